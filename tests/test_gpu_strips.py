"""Spatial decomposition with inactive bands (Sec. 6) on the GPU: R strips of
one system, each a library strip handle (hdmc_strip_*) with its own rows
and halo rows, swept through the strip protocol on one GPU, must follow the
serial banded oracle bit for bit (positions, slot order and counts of every
strip's own rows, the summed trial counters and the summed contact
histogram), in both precisions.
"""
import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import strips as S
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PREC = {"fp64": O.FP64, "fp32": O.FP32}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("R", [1, 2, 3, 5])
def test_strips_follow_the_serial_banded_chain(prec, R):
    w = W.n65536_phi070()
    strips = [S.Strip(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 7, prec, R, k) for k in range(R)]
    run = S.StripRun(strips, S.LocalExchange(strips))
    ref = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 7, PREC[prec])
    ref.set_strips(R)
    assert [(s.r0, s.r1) for s in strips] == ref.strip_rows(R)
    for n in (4, 16):
        run.sweep(n)
        ref.sweep(n)
        loc, cnt = ref.state()
        loc = loc.reshape(ref.my, ref.mx, 4, 2)
        cnt = cnt.reshape(ref.my, ref.mx)
        for s in strips:
            l, c = s.own_state()
            assert np.array_equal(c, cnt[s.r0:s.r1]), (R, s.strip)
            assert np.array_equal(l, loc[s.r0:s.r1]), (R, s.strip)
    assert np.array_equal(sum(s.counters() for s in strips), ref.counters())
    run.sample()
    hist, ns = run.histogram()
    assert ns == 1 and np.array_equal(hist, ref.histogram(200, 1e-4))
    for s in strips:
        s.close()


def test_strip_pressure_is_the_whole_system_fit():
    from paper_1211_1646_gb300 import hdmc
    from oracle import pressure as P
    w = W.n65536_phi070()
    strips = [S.Strip(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 3, "fp64", 4, k) for k in range(4)]
    run = S.StripRun(strips, S.LocalExchange(strips))
    ref = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 3, O.FP64)
    ref.set_strips(4)
    run.sweep(10)
    ref.sweep(10)
    run.sample()
    bp, g0 = run.pressure(w.N, w.Lx, w.Ly)
    bp_ref, g0_ref, _ = P.pressure(ref.histogram(200, 1e-4), 1, w.N, w.Lx * w.Ly)
    assert abs(bp - bp_ref) < 1e-9 * bp_ref and abs(g0 - g0_ref) < 1e-9 * g0_ref
    # whole-system entry points refuse a strip handle
    with pytest.raises(hdmc.HDMCError):
        hdmc.hdmc_sweep(strips[0].h, 1)
    with pytest.raises(hdmc.HDMCError):
        hdmc.hdmc_strip_shift(strips[0].h)   # phase 2 before phase 1
    for s in strips:
        s.close()
