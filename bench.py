#!/usr/bin/env python
"""Throughput of the checkerboard hard-disk Monte Carlo sweep on GB300.

Workload (synthetic, generated here): N = 1024^2 hard disks of diameter 1 in
the periodic box of a 1024 x 1024 hexagonal patch at packing fraction
phi = 0.716 (1152.45 x 998.06), hexagonal start with 0.01 sigma jitter,
maximum displacement d = 0.08 sigma, n_M = 4 trial moves per cell and
sub-sweep.  One step = 100 sweeps (Alg. 1: 4 sub-sweeps + 1 cell shift each)
+ one contact histogram + the pressure fit (Sec. 4), i.e. every stage of the
hot path.  Metric: attempted trial moves per second (Sec. 5.1), counted by
the library's trial counters, for the binary32 cell-local path; the binary64
path is timed on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hdmc|reference]

With torchrun (N > 1) every rank runs an independent replica (seed 1+rank);
the value is the sum of trial moves over ranks divided by the slowest
rank's time ("replicas only": the method has no cross-replica exchange).
--impl reference times the CPU oracle (all host cores) on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SWEEPS_PER_STEP = 100
METRIC = "trial moves/sec at N=1M phi=0.716 (1 GB300), FP32-local vs FP64; % HBM roofline"
KERNELS_PER_SWEEP = 5          # 4 sub-sweeps + 1 cell shift
SPHERE_KERNELS_PER_SWEEP = 9   # 8 sub-sweeps + 1 cell shift (three dimensions)
GRAPH_CHUNK = 64               # sweeps per recorded graph (one draws kernel each)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hdmc", choices=["hdmc", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the binary64 path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-replica batch leg")
    ap.add_argument("--no-n4m", action="store_true", help="skip the N=4M legs")
    ap.add_argument("--no-paper", action="store_true", help="skip the leg on the paper's Table 4 workload")
    ap.add_argument("--no-spheres", action="store_true", help="skip the hard-sphere (3-d) legs")
    ap.add_argument("--ncu-case", default=None, choices=["n1m", "n4m", "spheres", "batch64", "table4"],
                    help="run a short fixed workload for an ncu capture and exit (no timing)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    return ap.parse_args()


def ncu_case(args):
    """A few sweeps and one contact histogram of the N=1M (74 MB of binary32
    state) or N=4M (294 MB, larger than L2) phi=0.716 workload, of the
    paper's Table 4 workload, of the 64-replica batch or of the spheres."""
    import torch
    from paper_1211_1646_gb300 import build, hdmc, workloads
    build.build()
    if args.ncu_case == "batch64":
        b = hdmc.Batch(workloads.batch64(), precision="fp32")
        b.set_rows(1)
        hdmc.hdmc_batch_set_nselect(b.b, [8] * b.R)   # the autotuner's choice for this workload
        b.sweep(3)
        b.sample()
        b.pressure()
        torch.cuda.synchronize()
        print("ncu case batch64 done: %d replicas, %d disks" % (b.R, sum(b.N)))
        return
    if args.ncu_case == "spheres":
        w = workloads.spheres_n1m_phi049(args.precision)
        s = hdmc.System3(w.N, w.L, 1.0, w.d, w.nselect, 1, args.precision)
        s.sweep(3)
        s.sample()
        s.pressure()
        torch.cuda.synchronize()
        print("ncu case %s %s done: counters %s" % (w.name, args.precision, list(s.counters())))
        return
    if args.ncu_case == "table4":
        w = workloads.paper_table4()
        s = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 1, args.precision, cells="sqrt2")
    else:
        w = workloads.n1m_phi0716() if args.ncu_case == "n1m" else workloads.n4m(0.716)
        s = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 1, args.precision)
    s.sweep(3)
    s.sample()
    s.pressure()
    torch.cuda.synchronize()
    print("ncu case %s %s done: counters %s" % (w.name, args.precision, list(s.counters())))


def workload():
    from paper_1211_1646_gb300 import workloads
    return workloads.n1m_phi0716("fp32")


SUBSWEEP_SOURCES = ("hdmc_device.cuh", "hdmc_common.cuh", "hdmc_subsweep.cuh")


SPHERE_SOURCES = ("hdmc_device.cuh", "hdmc_common.cuh", "hdmc3_device.cuh", "hdmc3_subsweep.cuh")


def subsweep_source_hash(sources=SUBSWEEP_SOURCES):
    """First 16 hex digits of the SHA-256 of a kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1211_1646_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary="subsweep_f32_n1m.md", sources=SUBSWEEP_SOURCES):
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    summary, or None when the kernel's sources changed since the capture."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        src_hash = subsweep_source_hash(sources)
    except OSError:
        return None
    t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    h = re.search(r"kernel_source_sha256_16:\s*(\w+)", text)
    if not t or not h or h.group(1) != src_hash:
        return None
    return int(t.group(1))


def profiled_traffic_spheres():
    return profiled_traffic("subsweep3_f32_n1m.md", SPHERE_SOURCES)


# ALU work of one binary32 hard-sphere trial move, in 32-bit lane operations
# (an FMA is one): the direction (Philox4x32-10 at 80 operations per block,
# two attempts per block; per attempt 12 for three 21-bit fields and their
# conversion, 4 for the ball test; 6/pi attempts per kept direction); trial
# position and containment (3 FMAs, 6 compares); the other spheres of the
# cell (0.37 on average, 7 each); the gathered candidates (12.5 on average at
# n_M = 4, about 11 tested before a hit ends the scan, 7 each); the cell's
# gather shared by its n_M = 4 trials (31 occupied neighbour slots at 13
# each, reach box 20); the shuffle shared likewise (a Philox block and the
# decode for the 27 % of cells with n >= 2).
SPHERE_ALU_OPS_PER_TRIAL = {
    "direction": (80.0 / 2 + 12 + 4) * 6 / math.pi,
    "trial_and_containment": 9.0,
    "own_cell": 0.37 * 7,
    "candidates": 11 * 7.0,
    "gather": (31 * 13 + 20) / 4.0,
    "shuffle": 0.27 * 100 / 4.0,
}

# ALU work of one binary32 disk trial move (Alg. 2), the method's own: the
# trial position against every other disk of the 3x3 cell neighbourhood, 5
# operations each (2 differences, 2 FMAs, 1 compare), for the mean number of
# such disks measured from the cell counts (live_candidates); trial coordinate and containment test, 2
# FMAs and 4 compares; the random stream, Philox4x32-10 at 80 operations per
# block (10 rounds of 2 wide multiplies = 4, 2 three-input XORs, 2 key
# additions) with 6 21-bit fields per block and 2 fields per attempt; 9
# operations per attempt for the direction (2 fields extracted, converted and
# scaled; u*u + v*v and its compare); 4/pi attempts per kept direction.
def alu_ops_per_trial(live_candidates):
    return {
        "candidate_tests": 5 * live_candidates,
        "trial_and_containment": 6,
        "philox": 80 * (4 / math.pi) / 3,
        "directions": 9 * (4 / math.pi),
    }


LANES_PER_SM = 128      # 32-bit ALU/FMA lanes per SM (4 partitions x 32)
MAX_SM_MHZ = 2070.0     # GB300 maximum SM clock


def live_candidates(sysm):
    """Mean number of other disks in the 3x3 cell neighbourhood of a disk
    (the overlap candidates of a trial move), from the system's cell counts:
    sum over disks of (disks in the 9 cells - 1) / N."""
    import numpy as np
    _, cnt = sysm.state()
    n = cnt.astype(np.int64).reshape(sysm.my, sysm.mx)
    nine = sum(np.roll(np.roll(n, dy, 0), dx, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    return float((n * (nine - 1)).sum() / n.sum())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=10)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_identifier(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return dev


class Ranks:
    """Rank plumbing of a replicas-only run (one process per GPU): each rank
    advances its own independent system; the only collectives are the
    barriers around the timed region and the reductions of the reported
    numbers (max of times, sum of work).  Without a process group every
    call is the identity."""

    def __init__(self, dist, device):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def replica_seed(rank):
    """Seed of rank r's independent replica."""
    return 1 + rank


def run_hdmc(args, rank, world, dist):
    import numpy as np
    import torch
    from paper_1211_1646_gb300 import build, hdmc, workloads

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    seed = replica_seed(rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2
    ranks = Ranks(dist, dev)
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    def one_step(sysm):
        sysm.sweep(SWEEPS_PER_STEP)
        sysm.sample()
        return sysm.pressure()[0]

    def sweeps_only(sysm):   # the paper's eta: sweeps alone (Sec. 5.1)
        sysm.sweep(SWEEPS_PER_STEP)
        return None

    def timed_steps(sysm, steps, warmup, sampler=None, step=None):
        step = step or one_step
        for _ in range(warmup):
            step(sysm)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        c0 = int(sysm.counters()[0])
        total_ms = 0.0
        pressures = []
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(steps):
                flush.fill_(1)                      # L2 flushed between timed steps (untimed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bp = step(sysm)
                e1.record(stream)
                e1.synchronize()
                total_ms += e0.elapsed_time(e1)
                pressures.append(bp)
        torch.cuda.synchronize(dev)
        barrier()
        trials = int(sysm.counters()[0]) - c0
        return trials, total_ms, pressures

    # ---- binary32 cell-local path (the headline) ----
    s32 = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, seed, "fp32", device=dev)
    sampler = ClockSampler(gpu_identifier(torch, local))
    trials, ms, press = timed_steps(s32, args.steps, args.warmup, sampler)
    ms_max = max_over_ranks(ms)
    trials_all = sum_over_ranks(trials)
    value = trials_all / (ms_max / 1e3)
    clocks = sampler.summary()

    # kernel-level times inside recorded graphs, as in the timed step (the
    # sub-sweeps of 128 sweeps without shifts, then 128 shifts), on the same
    # stream with CUDA events; and one launch at a time for comparison
    live = live_candidates(s32)
    ms_sub, ms_shift = hdmc.hdmc_profile_stages(s32.h, 128)
    ms_sub_iso, ms_shift_iso, ms_draw = hdmc.hdmc_profile_sweeps(s32.h, 20)
    hbm_peak, peak_kind = load_peaks()
    # algorithmic bytes of one sub-sweep launch: every live particle read once
    # (the halos of the active cells cover the grid) and the active set's
    # particles written once, 1.25 N x 8 B (binary32 offsets), plus the
    # occupancy count of every cell, C x 1 B
    bytes_sub = 1.25 * w.N * 8 + s32.mx * s32.my
    achieved_hbm = bytes_sub / (ms_sub / 1e3) / 1e9
    # ALU roofline: the state (8 floats per cell, 37 MB) stays in L2 through
    # a step, and the sub-sweep is bound by the lane-operation rate
    trials_per_launch = trials / args.steps / (SWEEPS_PER_STEP * 4)
    alu_ops = alu_ops_per_trial(live)
    ops_per_trial = sum(alu_ops.values())
    achieved_alu = ops_per_trial * trials_per_launch / (ms_sub / 1e3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or MAX_SM_MHZ
    alu_peak = sms * LANES_PER_SM * mhz * 1e6 / 1e12

    # ---- end to end through the C ABI with host buffers ----
    # Each step loads the system's snapshot from pinned host memory (H2D),
    # runs the step (its histogram and pressure come back to the host) and
    # writes the new snapshot back (D2H).
    snap = torch.empty(s32.snapshot_bytes(), dtype=torch.uint8, pin_memory=True)
    s32.save(snap)
    h2d = snap.numel()
    d2h = snap.numel() + 200 * 8
    e2e_trials, e2e_s = 0, 0.0
    torch.cuda.synchronize(dev)
    for k in range(max(1, args.steps)):
        c0 = int(s32.counters()[0])
        t0 = time.perf_counter()
        s32.load(snap)                        # H2D: the step's input state
        one_step(s32)                         # D2H: histogram -> pressure
        s32.save(snap)                        # D2H: the state after the step
        t1 = time.perf_counter()
        e2e_trials += int(s32.counters()[0]) - c0
        e2e_s += t1 - t0
    e2e_s = max_over_ranks(e2e_s)
    e2e_value = sum_over_ranks(e2e_trials) / e2e_s
    s32.close()

    # ---- binary64 path on the same workload ----
    s64 = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, seed, "fp64", device=dev)
    t64, ms64, _ = timed_steps(s64, args.fp64_steps, 1)
    ms64 = max_over_ranks(ms64)
    value64 = sum_over_ranks(t64) / (ms64 / 1e3)
    ms_sub64, ms_shift64 = hdmc.hdmc_profile_stages(s64.h, 8)
    s64.close()

    # ---- N = 2048^2 at the four densities of that workload (state larger than L2) ----
    n4m = None
    if not args.no_n4m:
        n4m = {}
        for phi in (0.700, 0.710, 0.716, 0.720):
            w4 = workloads.n4m(phi)
            s4 = hdmc.System(w4.N, w4.Lx, w4.Ly, 1.0, w4.d, w4.nselect, seed, "fp32", device=dev)
            t4, ms4, _ = timed_steps(s4, args.steps, max(1, args.warmup))
            ms4 = max_over_ranks(ms4)
            sub4, shift4 = hdmc.hdmc_profile_stages(s4.h, 64)
            bytes4 = 1.25 * w4.N * 8 + s4.mx * s4.my
            bytes4_shift = 2 * w4.N * 8 + 2 * s4.mx * s4.my
            n4m["%.3f" % phi] = {
                "value": sum_over_ranks(t4) / (ms4 / 1e3), "unit": "trial moves/s",
                "ms_per_step": ms4 / args.steps, "subsweep_ms": sub4, "shift_ms": shift4,
                "roofline_hbm_frac": bytes4 / (sub4 / 1e3) / 1e9 / hbm_peak,
                "shift_roofline_hbm_frac": bytes4_shift / (shift4 / 1e3) / 1e9 / hbm_peak}
            s4.close()

    # ---- the paper's own throughput workload (Sec. 5.1, Table 4): N = 1520^2,
    # phi = 0.698, cells just below sqrt(2) sigma; eta = trial moves of the
    # sweeps alone per second, for comparison with the paper's K20 figure ----
    paper = None
    if not args.no_paper:
        wp = workloads.paper_table4()
        sp = hdmc.System(wp.N, wp.Lx, wp.Ly, 1.0, wp.d, wp.nselect, seed, "fp32", device=dev, cells="sqrt2")
        tp, msp, _ = timed_steps(sp, args.steps, max(1, args.warmup), step=sweeps_only)
        msp = max_over_ranks(msp)
        paper = {"workload": wp.name, "N": wp.N, "phi": wp.phi, "cells": [sp.mx, sp.my], "d": wp.d,
                 "nselect": wp.nselect, "step": "%d sweeps" % SWEEPS_PER_STEP,
                 "value": sum_over_ranks(tp) / (msp / 1e3), "unit": "trial moves/s", "ms_per_step": msp / args.steps,
                 "disk_sweeps_per_s": sum_over_ranks(wp.N * SWEEPS_PER_STEP * args.steps) / (msp / 1e3),
                 "paper_value": 1.09e9, "paper_hardware": "Tesla K20, FP32, the same workload (Table 4)"}
        sp.close()

    # ---- 64 batched replicas of uneven N and phi in one launch per stage ----
    batch = None
    if not args.no_batch:
        reps = workloads.batch64()
        b = hdmc.Batch(reps, precision="fp32", device=dev)
        rows, nm = b.autotune(16)
        for _ in range(max(1, args.warmup)):
            one_step(b)
        torch.cuda.synchronize(dev)
        c0 = int(b.counters()[:, 0].sum())
        ms_b = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(b)
            e1.record(stream)
            e1.synchronize()
            ms_b += e0.elapsed_time(e1)
        tb = int(b.counters()[:, 0].sum()) - c0
        ms_b = max_over_ranks(ms_b)
        n_total = sum(r.N for r in reps)
        c_total = sum(int(gr["mx"]) * int(gr["my"]) for gr in b.grids)
        # whole-step roofline: per sweep every disk is read once per sub-sweep
        # and written once, the shift reads and writes it once, and the counts
        # are read 5 times and written once: 6 N x 8 B + 6 C x 1 B
        bytes_step = SWEEPS_PER_STEP * (6 * n_total * 8 + 6 * c_total)
        ach_b = bytes_step / (ms_b / args.steps / 1e3) / 1e9
        batch = {"value": sum_over_ranks(tb) / (ms_b / 1e3), "unit": "trial moves/s",
                 "disk_sweeps_per_s": n_total * SWEEPS_PER_STEP / (ms_b / args.steps / 1e3),
                 "ms_per_step": ms_b / args.steps, "replicas": len(reps), "N_total": n_total,
                 "rows_per_block": rows, "nselect": nm,
                 "roofline_step": {"bound": "hbm", "achieved": ach_b, "peak": hbm_peak, "unit": "GB/s",
                                   "frac": ach_b / hbm_peak, "peak_kind": peak_kind,
                                   "algorithmic_bytes_per_step": bytes_step},
                 "workload": "64 replicas, N log-uniform in [4096, 262144], phi uniform in [0.60, 0.74], "
                             "d = 0.08, autotuned (16 sweeps per candidate)"}
        b.close()

    # ---- hard spheres (three dimensions): N = 4*64^3 at phi = 0.49 ----
    spheres = None
    if not args.no_spheres:
        w3 = workloads.spheres_n1m_phi049("fp32")
        spheres = {"workload": w3.name, "N": w3.N, "phi": w3.phi, "box": [round(x, 4) for x in w3.L],
                   "d": w3.d, "nselect": w3.nselect, "unit": "trial moves/s",
                   "step": "%d sweeps (8 sub-sweeps + 1 shift each) + contact histogram + pressure fit"
                           % SWEEPS_PER_STEP,
                   "launches_per_step": SPHERE_KERNELS_PER_SWEEP * SWEEPS_PER_STEP
                                        + math.ceil(SWEEPS_PER_STEP / GRAPH_CHUNK) + 1}
        for prec, nsteps in (("fp32", args.steps), ("fp64", max(1, args.fp64_steps - 1))):
            s3 = hdmc.System3(w3.N, w3.L, 1.0, w3.d, w3.nselect, seed, prec)
            t3, ms3, p3 = timed_steps(s3, nsteps, 1)
            ms3 = max_over_ranks(ms3)
            sub3, shift3 = s3.profile_stages(16)   # in-step: runs of sub-sweeps / shifts, as in the step
            # algorithmic bytes of one sub-sweep launch, live data only: every
            # sphere read once (the neighbourhoods of the active cells cover
            # the grid) and the active set's spheres (one eighth) written
            # once, 3 coordinates of 4 B (binary32) or 8 B (binary64) each
            bytes3 = 1.125 * w3.N * 3 * (4 if prec == "fp32" else 8)
            ach = bytes3 / (sub3 / 1e3) / 1e9
            leg = {"value": sum_over_ranks(t3) / (ms3 / 1e3), "ms_per_step": ms3 / nsteps, "steps": nsteps,
                   "subsweep_ms": sub3, "shift_ms": shift3, "betaP_over_rho_last": p3[-1] if p3 else None}
            if prec == "fp32":
                leg["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                                   "frac": ach / hbm_peak, "traffic": profiled_traffic_spheres(),
                                   "kernel": "k_sub3<float>", "peak_kind": peak_kind,
                                   "ms_per_launch": sub3, "ms_per_launch_note": "in-step: mean over a run of "
                                   "sub-sweep launches", "algorithmic_bytes_per_launch": bytes3}
                tpl3 = t3 / nsteps / (SWEEPS_PER_STEP * 8)
                ops3 = sum(SPHERE_ALU_OPS_PER_TRIAL.values())
                ach3 = ops3 * tpl3 / (sub3 / 1e3) / 1e12
                leg["roofline_alu"] = {"bound": "alu", "achieved": ach3, "peak": alu_peak, "unit": "Tops/s",
                                       "frac": ach3 / alu_peak, "kernel": "k_sub3<float>",
                                       "trials_per_launch": tpl3, "ops_per_trial": ops3}
            if prec == "fp32":
                # end to end through the C ABI with host buffers: every step
                # loads the snapshot from pinned host memory (H2D), runs the
                # step (histogram back for the fit) and saves it (D2H)
                snap = torch.empty(s3.snapshot_bytes(), dtype=torch.uint8, pin_memory=True)
                s3.save(snap)
                e2e_t, e2e_s = 0, 0.0
                torch.cuda.synchronize(dev)
                for _ in range(max(1, nsteps)):
                    c0 = int(s3.counters()[0])
                    t0 = time.perf_counter()
                    s3.load(snap)
                    one_step(s3)
                    s3.save(snap)
                    e2e_s += time.perf_counter() - t0
                    e2e_t += int(s3.counters()[0]) - c0
                e2e_s = max_over_ranks(e2e_s)
                leg["e2e"] = {"value": sum_over_ranks(e2e_t) / e2e_s, "unit": "trial moves/s",
                              "h2d_bytes_per_step": snap.numel(), "d2h_bytes_per_step": snap.numel() + 200 * 8}
            spheres[prec] = leg
            s3.close()
        spheres["value"] = spheres["fp32"]["value"]
        spheres["e2e"] = spheres["fp32"]["e2e"]

    launches_per_step = KERNELS_PER_SWEEP * SWEEPS_PER_STEP + math.ceil(SWEEPS_PER_STEP / GRAPH_CHUNK) + 1
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "trial moves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "phi": 0.716, "box": [round(w.Lx, 4), round(w.Ly, 4)],
                   "cells": [s32.mx, s32.my], "d": w.d, "nselect": w.nselect,
                   "step": "%d sweeps + contact histogram + pressure fit" % SWEEPS_PER_STEP,
                   "trial_moves_per_step": trials / args.steps,
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas x%d" % world},
        "e2e": {"value": e2e_value, "unit": "trial moves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "disk_sweeps_per_s": sum_over_ranks(w.N * SWEEPS_PER_STEP * args.steps) / (ms_max / 1e3),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "roofline": {"bound": "hbm", "achieved": achieved_hbm, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_hbm / hbm_peak, "traffic": profiled_traffic(), "kernel": "k_subsweep_f32",
                     "traffic_note": "ncu dram bytes per launch inside a run of sweeps (no cache flush)",
                     "peak_kind": peak_kind, "ms_per_launch": ms_sub,
                     "ms_per_launch_note": "in-step: mean over the sub-sweep launches of recorded graphs",
                     "algorithmic_bytes_per_launch": bytes_sub},
        "roofline_alu": {"bound": "alu", "achieved": achieved_alu, "peak": alu_peak, "unit": "Tops/s",
                         "frac": achieved_alu / alu_peak, "kernel": "k_subsweep_f32",
                         "peak_kind": "derived: %d SMs x %d lanes x %.0f MHz" % (sms, LANES_PER_SM, mhz),
                         "trials_per_launch": trials_per_launch, "ops_per_trial": ops_per_trial,
                         "live_candidates_per_trial": live},
        "kernels_ms": {"subsweep_f32": ms_sub, "shift_f32": ms_shift, "draws": ms_draw,
                       "subsweep_f32_one_launch": ms_sub_iso, "shift_f32_one_launch": ms_shift_iso,
                       "subsweep_f64": ms_sub64, "shift_f64": ms_shift64,
                       "note": "subsweep_f32/shift_f32: mean per launch inside recorded graphs (in-step); "
                               "*_one_launch and f64: one launch at a time"},
        "step_check_ms": {"subsweeps_plus_shifts": SWEEPS_PER_STEP * (4 * ms_sub + ms_shift),
                          "ms_per_step": ms_max / args.steps},
        "fp64": {"value": value64, "unit": "trial moves/s", "ms_per_step": ms64 / max(1, args.fp64_steps),
                 "steps": args.fp64_steps},
        "speedup_fp32_over_fp64": value / value64 if value64 > 0 else None,
        "batch64": batch,
        "n4m": n4m,
        "paper_table4": paper,
        "spheres": spheres,
        "pressure_betaP_over_rho_last": press[-1] if press else None,
    }
    return line


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def oracle_sample(seconds_budget=12.0, threads=None):
    """The oracle, as it stands, on the bench workload (binary32 mode, all
    host cores): sweeps + one contact histogram + the pressure fit, until the
    time budget is used.  Returns (trial moves/s, threads, description)."""
    import oracle
    w = workload()
    nt = oracle.set_threads(threads or (os.cpu_count() or 1))
    s = oracle.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 1, oracle.FP32)
    t0 = time.perf_counter()
    c0 = int(s.counters()[0])
    sweeps = 0
    while True:
        s.sweep(1)
        sweeps += 1
        if time.perf_counter() - t0 > seconds_budget * 0.8:
            break
    h = s.histogram()
    oracle.pressure.pressure(h, 1, w.N, w.Lx * w.Ly)
    dt = time.perf_counter() - t0
    trials = int(s.counters()[0]) - c0
    return trials / dt, nt, "%d sweeps + 1 contact histogram + pressure fit of the N=1048576 workload" % sweeps


def oracle_sample_spheres(seconds_budget=8.0, threads=None):
    """The oracle's three-dimensional form, as it stands, on the sphere
    workload (binary32 mode, all host cores): sweeps + one contact histogram
    + the pressure fit, until the time budget is used."""
    import oracle
    from paper_1211_1646_gb300 import workloads
    w = workloads.spheres_n1m_phi049("fp32")
    nt = oracle.set_threads(threads or (os.cpu_count() or 1))
    s = oracle.System3(w.N, w.L, 1.0, w.d, w.nselect, 1, oracle.FP32)
    t0 = time.perf_counter()
    c0 = int(s.counters()[0])
    sweeps = 0
    while True:
        s.sweep(1)
        sweeps += 1
        if time.perf_counter() - t0 > seconds_budget * 0.8:
            break
    h = s.histogram()
    oracle.pressure.pressure3(h, 1, w.N, w.L[0] * w.L[1] * w.L[2])
    dt = time.perf_counter() - t0
    trials = int(s.counters()[0]) - c0
    return trials / dt, nt, "%d sweeps + 1 contact histogram + pressure fit of the %d-sphere workload" % (sweeps, w.N)


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores, same workload."""
    import oracle
    w = workload()
    nt = oracle.set_threads(os.cpu_count() or 1)
    s = oracle.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 1, oracle.FP32)

    def step():   # the GPU arm's step: 100 sweeps + one contact histogram + the fit
        s.sweep(SWEEPS_PER_STEP)
        h = s.histogram()
        oracle.pressure.pressure(h, 1, w.N, w.Lx * w.Ly)

    for _ in range(args.warmup):
        step()
    c0 = int(s.counters()[0])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    trials = int(s.counters()[0]) - c0
    value = trials / dt
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "trial moves/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "phi": 0.716, "d": w.d, "nselect": w.nselect,
                   "step": "%d sweeps + contact histogram + pressure fit (CPU oracle)" % SWEEPS_PER_STEP},
        "cpu_baseline": {"value": value, "unit": "trial moves/s", "cores": nt, "kind": "oracle",
                         "sample": "%d steps of %d sweeps + contact histogram + pressure fit, N=1048576"
                                   % (args.steps, SWEEPS_PER_STEP)},
        "e2e": {"value": value, "unit": "trial moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    if args.ncu_case:
        ncu_case(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_hdmc(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            v, nt, sample = oracle_sample()
            v1, _, sample1 = oracle_sample(seconds_budget=6.0, threads=1)
            line["cpu_baseline"] = {"value": v, "unit": "trial moves/s", "cores": nt, "kind": "oracle",
                                    "sample": sample,
                                    "serial": {"value": v1, "unit": "trial moves/s", "cores": 1, "sample": sample1}}
            if line.get("spheres"):
                v3, nt3, sample3 = oracle_sample_spheres()
                line["spheres"]["cpu_baseline"] = {"value": v3, "unit": "trial moves/s", "cores": nt3,
                                                   "kind": "oracle", "sample": sample3}
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
