"""The multi-rank host logic of bench.py on CPU: two gloo ranks (processes
spawned on 127.0.0.1), no GPU.  With one replica per rank the only
collectives are barriers and the max / sum reductions of the reported
numbers."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = bench.Ranks(dist, torch.device("cpu"))
        r.barrier()
        res = {
            "max": r.max(10.0 * (rank + 1)),          # slowest rank's time
            "sum": r.sum(1000 * (rank + 1)),          # work of all ranks
            "seed": bench.replica_seed(rank),
        }
        r.barrier()
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_seed():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        assert got[rank]["max"] == 20.0
        assert got[rank]["sum"] == 3000.0
    assert got[0]["seed"] != got[1]["seed"]


def test_single_process_ranks_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(None, None)
    r.barrier()
    assert r.max(3.5) == 3.5 and r.sum(7) == 7


def test_reference_arm_prints_one_contract_line():
    # bench.py --impl reference runs the oracle on the host cores (no GPU)
    # and prints one JSON line with the keys of the bench contract
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "n1048576_phi0.716_hex"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
