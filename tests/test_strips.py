"""Spatial decomposition with inactive bands (Sec. 6) on CPU: the strip
protocol of paper_1211_1646_gb300.strips (which rows move between strips,
and when) driving oracle-backed strips, in one process and over two gloo
ranks, must reproduce the serial banded oracle bit for bit.

An OracleStrip is a whole banded oracle system of which only the strip's
own rows and its halo rows are kept: after every phase the other rows are
emptied, so what the strip knows of its neighbours comes from the rows the
protocol moves.  A missing or late row exchange shows up as a difference in
the own rows.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import strips as S
from paper_1211_1646_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleStrip:
    """Strip k of R backed by a whole banded oracle system (tests only)."""

    def __init__(self, w, seed, prec, R, k):
        self.o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, seed, prec)
        self.o.set_strips(R)
        self.r0, self.r1 = self.o.strip_rows(R)[k]
        self.mx, self.my = self.o.mx, self.o.my
        self._isolate()

    def row_buffer(self, host=False):
        import torch
        return torch.zeros(self.mx * 9, dtype=torch.float64)

    def _own(self, which):
        return [self.r0, self.r0 + 1, self.r1 - 2, self.r1 - 1][which]

    def _halo(self, which):
        return [self.r0 - 2, self.r0 - 1, self.r1, self.r1 + 1][which] % self.my

    def get_row(self, which, buf):
        loc, cnt = self.o.get_row(self._own(which))
        buf[: self.mx * 8] = __import__("torch").from_numpy(loc.reshape(-1))
        buf[self.mx * 8:] = __import__("torch").from_numpy(cnt.astype(np.float64))

    def set_halo(self, which, buf):
        b = buf.numpy()
        self.o.set_row(self._halo(which), b[: self.mx * 8].reshape(self.mx, 4, 2), b[self.mx * 8:].astype(np.uint8))

    def _isolate(self):
        keep = {r % self.my for r in range(self.r0 - 2, self.r1 + 2)}
        empty = np.full((self.mx, 4, 2), -1.0e4)
        zero = np.zeros(self.mx, dtype=np.uint8)
        for r in range(self.my):
            if r not in keep:
                self.o.set_row(r, empty, zero)

    def subsweeps(self):
        self.o.sweep_phase(0)
        self._isolate()

    def shift(self):
        self.o.sweep_phase(1)
        self._isolate()

    def sample(self):
        pass

    def own_rows(self):
        loc, cnt = self.o.state()
        loc = loc.reshape(self.my, self.mx, 4, 2)[self.r0:self.r1]
        cnt = cnt.reshape(self.my, self.mx)[self.r0:self.r1]
        return loc, cnt


def _serial(w, seed, prec, R, sweeps):
    o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, seed, prec)
    o.set_strips(R)
    o.sweep(sweeps)
    loc, cnt = o.state()
    return o, loc.reshape(o.my, o.mx, 4, 2), cnt.reshape(o.my, o.mx)


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
@pytest.mark.parametrize("R", [1, 2, 3])
def test_protocol_reproduces_the_serial_banded_chain(prec, R):
    w = W.n1024_phi070()
    strips = [OracleStrip(w, 11, prec, R, k) for k in range(R)]
    run = S.StripRun(strips, S.LocalExchange(strips))
    run.sweep(30)
    o, loc, cnt = _serial(w, 11, prec, R, 30)
    for s in strips:
        l, c = s.own_rows()
        assert np.array_equal(c, cnt[s.r0:s.r1]), (R, s.r0)
        assert np.array_equal(l, loc[s.r0:s.r1]), (R, s.r0)


@pytest.mark.parametrize("dropped", ["LAST_TO_NEXT", "BAND_TO_PREV"])
def test_a_missing_exchange_is_detected(dropped):
    # without the row sent before the shift, migrants of a -y shift enter
    # the strip from a stale row; without the band row sent after it, the
    # strip keeps its own (stale) copy of the next strip's band row, whose
    # errors reach the own rows within a few tens of sweeps
    w = W.n1024_phi070()
    R = 2
    strips = [OracleStrip(w, 11, O.FP64, R, k) for k in range(R)]
    run = S.StripRun(strips, S.LocalExchange(strips))
    moves = getattr(S, dropped)
    saved = moves[:]
    try:
        moves.clear()
        run.sweep(80)
    finally:
        moves[:] = saved
    _, loc, cnt = _serial(w, 11, O.FP64, R, 80)
    same = all(np.array_equal(s.own_rows()[0], loc[s.r0:s.r1]) for s in strips)
    assert not same


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, prec, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.n1024_phi070()
        s = OracleStrip(w, 5, prec, world, rank)
        run = S.StripRun([s], S.DistExchange(s, dist, rank, world, host=True))
        run.sweep(25)
        _, loc, cnt = _serial(w, 5, prec, world, 25)
        l, c = s.own_rows()
        out.put((rank, bool(np.array_equal(l, loc[s.r0:s.r1]) and np.array_equal(c, cnt[s.r0:s.r1]))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_two_gloo_ranks_reproduce_the_serial_banded_chain(prec):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, prec, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == {0: True, 1: True}
