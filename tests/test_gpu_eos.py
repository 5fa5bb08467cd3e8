"""Equation of state: the binary32 path and batched binary32 replicas against
the binary64 path (statistical comparison).

The three paths follow different trajectories (different arithmetic), so only
their pressures can be compared.  The Sec. 4 estimator extrapolates a
degree-5 fit to contact, whose relative noise is about 6/sqrt(pair counts),
so each path collects ~10^10 contact pairs (10^6 disks, 6000 samples) at a
liquid state point, for a block-averaged standard error of P* near 1e-4
relative; the binary32 results must agree with binary64 within
|dP|/P <= 5e-4 and within 3 combined standard errors.
"""
import math

import numpy as np
import pytest

from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PHI = 0.66
SWEEPS = 60_000
EVERY = 10
BLOCKS = 12
EQUIL = 4000


def _pstar(bp, N, area):
    return bp * N / area   # P* = rho sigma^2 (beta P / rho), sigma = 1


def _run_blocks(advance, pressure, N, area):
    """Block averages of P*: each block accumulates SWEEPS/BLOCKS/EVERY histograms."""
    per_block = SWEEPS // BLOCKS // EVERY
    out = []
    for _ in range(BLOCKS):
        for _ in range(per_block):
            advance(EVERY)
        out.append(pressure())
    return np.array(out)


def _mean_se(x):
    return x.mean(), x.std(ddof=1) / math.sqrt(len(x))


@pytest.mark.slow
def test_fp32_and_batched_pressure_match_fp64():
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    nx = ny = 1024
    Lx, Ly = W.hex_box(nx, ny, PHI)
    N, area = nx * ny, Lx * Ly

    # binary64 reference, equilibrated from the hexagonal start
    s64 = hdmc.System(N, Lx, Ly, 1.0, 0.1, 4, 101, "fp64")
    s64.sweep(EQUIL)
    loc, cnt = s64.state()
    info = s64.info()

    # binary32 system continuing from the same configuration (rounded to binary32)
    s32 = hdmc.System(N, Lx, Ly, 1.0, 0.1, 4, 202, "fp32")
    wx32, wy32 = np.float32(s32.wx), np.float32(s32.wy)
    l32 = loc.astype(np.float32)
    occ = np.arange(4)[None, :] < cnt[:, None]
    l32[..., 0] = np.where(occ, np.minimum(l32[..., 0], np.nextafter(wx32, 0)), l32[..., 0])
    l32[..., 1] = np.where(occ, np.minimum(l32[..., 1], np.nextafter(wy32, 0)), l32[..., 1])
    s32.set_state(l32.astype(np.float64), cnt, info["origin"], 0, 0)

    # four batched binary32 replicas at the same state point, own equilibration
    reps = [W.Workload("r%d" % k, N, Lx, Ly, 0.1, 4, 300 + k, 0) for k in range(4)]
    bat = hdmc.Batch(reps, precision="fp32")
    bat.sweep(EQUIL)

    def adv_sample(sys_):
        def f(n):
            sys_.sweep(n)
            sys_.sample()
        return f

    p64 = _run_blocks(adv_sample(s64), lambda: _pstar(s64.pressure()[0], N, area), N, area)
    p32 = _run_blocks(adv_sample(s32), lambda: _pstar(s32.pressure()[0], N, area), N, area)
    per_block = SWEEPS // BLOCKS // EVERY // 4   # the batch has 4x the disks per sample
    pb = []
    for _ in range(BLOCKS):
        for _ in range(per_block):
            bat.sweep(EVERY)
            bat.sample()
        bp, _, _, _ = bat.pressure()
        pb.append(float(np.mean(_pstar(bp, N, area))))
    pb = np.array(pb)
    torch.cuda.synchronize()

    m64, e64 = _mean_se(p64)
    for name, p in (("fp32", p32), ("batched fp32", pb)):
        m, e = _mean_se(p)
        diff = abs(m - m64)
        comb = math.sqrt(e * e + e64 * e64)
        print("%s: P* = %.5f +- %.5f vs fp64 %.5f +- %.5f (|dP|/P = %.2e, %.2f SE)"
              % (name, m, e, m64, e64, diff / m64, diff / comb))
        assert diff / m64 <= 5e-4, name
        assert diff <= 3 * comb, name
    # the statistics are fine enough for the tolerance to mean something
    assert e64 / m64 < 2e-4


def _to_fp32(loc, cnt, wx, wy):
    """binary64 local coordinates rounded to binary32, kept below the binary32 widths."""
    wx32, wy32 = np.float32(wx), np.float32(wy)
    l32 = loc.astype(np.float32)
    occ = np.arange(4)[None, :] < cnt[:, None]
    l32[..., 0] = np.where(occ, np.minimum(l32[..., 0], np.nextafter(wx32, 0)), l32[..., 0])
    l32[..., 1] = np.where(occ, np.minimum(l32[..., 1], np.nextafter(wy32, 0)), l32[..., 1])
    return l32.astype(np.float64)


def _to_fp64(loc, cnt, wx, wy):
    """binary32 local coordinates (exact in binary64) kept below the binary64 widths."""
    out = loc.copy()
    occ = np.arange(4)[None, :] < cnt[:, None]
    out[..., 0] = np.where(occ, np.minimum(out[..., 0], np.nextafter(wx, 0)), out[..., 0])
    out[..., 1] = np.where(occ, np.minimum(out[..., 1], np.nextafter(wy, 0)), out[..., 1])
    return out


def _paired(p, p64):
    """Mean and standard error of the block-wise differences p - p64 of two
    runs from one start over the same sweeps (a drift common to both, as
    from a start that is still relaxing, cancels in the differences)."""
    d = np.asarray(p) - np.asarray(p64)
    return d.mean(), d.std(ddof=1) / math.sqrt(len(d))


@pytest.mark.slow
def test_fp32_and_batched_pressure_match_fp64_at_the_benchmark_state_point():
    # N = 1024^2 at phi = 0.716 (the state point of the throughput benchmark,
    # in the liquid-hexatic coexistence range, where the pressure relaxes
    # slowly): 2 10^5 binary32 sweeps from the hexagonal start, then binary64,
    # binary32 and four batched binary32 replicas continue from that one
    # configuration with the same random streams (seed and sweep index;
    # replicas 1-3 with their own seeds) for 6 10^4 sweeps.  The Sec. 4
    # pressures of the block-wise differences agree within |dP|/P <= 5e-4 and
    # 3 standard errors.
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    w = W.n1m_phi0716("fp32")
    N, area = w.N, w.Lx * w.Ly
    equil = 200_000
    s32 = hdmc.System(N, w.Lx, w.Ly, 1.0, w.d, 4, 101, "fp32")
    s32.sweep(equil)
    loc, cnt = s32.state()
    info = s32.info()
    s64 = hdmc.System(N, w.Lx, w.Ly, 1.0, w.d, 4, 101, "fp64")
    s64.set_state(_to_fp64(loc, cnt, s64.wx, s64.wy), cnt, info["origin"], info["sweeps_done"],
                  info["shifts_done"])
    reps = [W.Workload("r%d" % k, N, w.Lx, w.Ly, w.d, 4, 101 + k, 0) for k in range(4)]
    bat = hdmc.Batch(reps, precision="fp32")
    for r in range(4):
        bat.set_state(r, loc, cnt, info["origin"], info["sweeps_done"])

    def adv_sample(sys_):
        def f(n):
            sys_.sweep(n)
            sys_.sample()
        return f

    p64 = _run_blocks(adv_sample(s64), lambda: _pstar(s64.pressure()[0], N, area), N, area)
    p32 = _run_blocks(adv_sample(s32), lambda: _pstar(s32.pressure()[0], N, area), N, area)
    per_block = SWEEPS // BLOCKS // EVERY
    pb = []
    for _ in range(BLOCKS):
        for _ in range(per_block):
            bat.sweep(EVERY)
            bat.sample()
        bp, _, _, _ = bat.pressure()
        pb.append(float(np.mean(_pstar(bp, N, area))))
    pb = np.array(pb)
    torch.cuda.synchronize()
    m64, e64 = _mean_se(p64)
    for name, p in (("fp32", p32), ("batched fp32", pb)):
        m, e = _mean_se(p)
        dm, de = _paired(p, p64)
        print("phi 0.716 %s: P* = %.5f +- %.5f vs fp64 %.5f +- %.5f; paired difference %.5f +- %.5f "
              "(|dP|/P = %.2e, %.2f SE)" % (name, m, e, m64, e64, dm, de, abs(dm) / m64, abs(dm) / de))
        assert abs(dm) / m64 <= 5e-4, name
        assert abs(dm) <= 3 * de, name


@pytest.mark.slow
def test_fp32_runs_match_fp64_on_overlap_windows_at_4m():
    # N = 2048^2 at phi = 0.700, 0.710, 0.716, 0.720: binary32 runs of 2 10^4
    # sweeps from the hexagonal start, then a 10^3-sweep window in which a
    # binary64 system continues from the binary32 configuration (same seed,
    # same sweep index); the block-wise pressure differences over the window
    # agree within |dP|/P <= 5e-4 and 3 standard errors.
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    window, every, blocks = 1000, 10, 10
    for phi in (0.700, 0.710, 0.716, 0.720):
        w = W.n4m(phi)
        N, area = w.N, w.Lx * w.Ly
        s32 = hdmc.System(N, w.Lx, w.Ly, 1.0, w.d, 4, 7, "fp32")
        s32.sweep(20_000)
        loc, cnt = s32.state()
        info = s32.info()
        s64 = hdmc.System(N, w.Lx, w.Ly, 1.0, w.d, 4, 7, "fp64")
        s64.set_state(_to_fp64(loc, cnt, s64.wx, s64.wy), cnt, info["origin"], info["sweeps_done"],
                      info["shifts_done"])
        res = {}
        for name, s in (("fp32", s32), ("fp64", s64)):
            out = []
            for _ in range(blocks):
                for _ in range(window // blocks // every):
                    s.sweep(every)
                    s.sample()
                out.append(_pstar(s.pressure()[0], N, area))
            res[name] = np.array(out)
            s.close()
        torch.cuda.synchronize()
        (m32, e32), (m64, e64) = _mean_se(res["fp32"]), _mean_se(res["fp64"])
        dm, de = _paired(res["fp32"], res["fp64"])
        print("N=2048^2 phi %.3f: fp32 P* = %.5f +- %.5f, fp64 %.5f +- %.5f; paired difference %.5f +- %.5f "
              "(|dP|/P = %.2e, %.2f SE)" % (phi, m32, e32, m64, e64, dm, de, abs(dm) / m64, abs(dm) / de))
        assert abs(dm) / m64 <= 5e-4, phi
        assert abs(dm) <= 3 * de, phi

