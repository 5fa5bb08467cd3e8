"""Parity of the CUDA library's three-dimensional (hard-sphere) path with the
oracle, through the C ABI.

Both are deterministic functions of (configuration, seed, sweep index): the
binary64 and binary32 paths must agree with the oracle's modes bit for bit
-- local coordinates, cell counts, slot order, trial counters, grid origin
and the contact histogram.  Sizes run from a single sphere to the N = 1M
benchmark workload (checked after a few sweeps against the multi-threaded
oracle), with ragged last blocks and cells holding up to eight spheres.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
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
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


def _pair(N, L, prec, d=0.1, nsel=4, seed=1, xyz=None):
    from paper_1211_1646_gb300 import hdmc
    g = hdmc.System3(N, L, 1.0, d, nsel, seed, prec, xyz=xyz)
    o = O.System3(N, L, 1.0, d, nsel, seed, PREC[prec], xyz=xyz)
    return g, o


def _same(g, o):
    gl, gc = g.state()
    ol, oc = o.state()
    assert np.array_equal(gc, oc)
    assert np.array_equal(gl, ol)
    assert np.array_equal(g.counters(), o.counters())
    assert np.array_equal(g.origin(), o.origin())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_start_state_matches(prec):
    w = W.spheres_n2048_phi045()
    g, o = _pair(w.N, w.L, prec, w.d)
    _same(g, o)
    assert np.array_equal(g.positions(), o.positions())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case,sweeps", [("n2048", 25), ("n16384", 6)])
def test_sweeps_bit_identical(prec, case, sweeps):
    w = W.spheres_n2048_phi045() if case == "n2048" else W.spheres_n16384_phi045()
    g, o = _pair(w.N, w.L, prec, w.d, seed=11)
    g.sweep(sweeps)
    o.sweep(sweeps)
    _same(g, o)
    assert np.array_equal(g.positions(), o.positions())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_each_subsweep_and_explicit_shifts(prec):
    w = W.spheres_n2048_phi045()
    g, o = _pair(w.N, w.L, prec, w.d, nsel=7, seed=12)
    for Q in (5, 0, 7, 2, 3, 6, 1, 4):
        g.subsweep(900 + Q, Q)
        o.subsweep(900 + Q, Q)
        _same(g, o)
    for _ in range(7):
        g.shift()
        o.shift()
    _same(g, o)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_histogram_matches(prec):
    w = W.spheres_n2048_phi045()
    g, o = _pair(w.N, w.L, prec, w.d, seed=13)
    g.sweep(20)
    o.sweep(20)
    g.sample()
    _, _, hist, ns = g.pressure()
    assert ns == 1
    ref = o.histogram(200, 1e-4)
    assert ref.sum() > 100 and np.array_equal(hist, ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_balance_controls_match(prec):
    w = W.spheres_n2048_phi045()
    for sp, ss in ((False, True), (True, False), (False, False)):
        g, o = _pair(w.N, w.L, prec, w.d, seed=14)
        g.set_balance(sp, ss)
        o.set_balance(sp, ss)
        g.sweep(8)
        o.sweep(8)
        _same(g, o)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eight_spheres_in_one_cell(prec):
    # a cell at full occupancy (eight spheres near its corners), the rest empty
    w = 1.1
    xyz = 0.01 + np.array(list(itertools.product([0.0, 1.05], repeat=3)))
    g, o = _pair(8, [4 * w] * 3, prec, d=0.3, nsel=16, seed=15, xyz=xyz)
    assert g.state()[1].max() == 8
    g.sweep(30)
    o.sweep(30)
    _same(g, o)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_sphere_and_uneven_box(prec):
    g, o = _pair(1, [4.4, 5.1, 6.3], prec, d=0.4, nsel=3, seed=16, xyz=np.array([[1.0, 2.0, 3.0]]))
    g.sweep(40)
    o.sweep(40)
    _same(g, o)
    # an uneven box with many cells per axis and a ragged last block
    L = [13.3, 10.6, 11.9]
    xyz = O.lattice3_positions(4 * 6**3, [13.3, 13.3, 13.3], 1.0, 3) * (np.array(L) / 13.3)
    g, o = _pair(len(xyz), L, prec, d=0.1, nsel=5, seed=17, xyz=xyz)
    g.sweep(10)
    o.sweep(10)
    _same(g, o)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_n1m_full_size_parity(prec):
    # the benchmark workload (N = 4*64^3, phi = 0.49), two sweeps
    w = W.spheres_n1m_phi049(prec)
    g, o = _pair(w.N, w.L, prec, w.d, w.nselect, w.seed)
    g.sweep(2)
    o.sweep(2)
    _same(g, o)
    c = g.counters()
    assert c[0] > 4 * 0.6 * w.N and 0.2 < c[1] / c[0] < 0.9


def test_errors():
    from paper_1211_1646_gb300 import hdmc
    w = W.spheres_n2048_phi045()
    for args in ((w.N, w.L, 1.0, 0.6), (w.N, [13.9] * 3, 1.0, 0.1), (2000, w.L, 1.0, 0.1), (w.N, [3.9] * 3, 1.0, 0.1)):
        with pytest.raises(hdmc.HDMCError) as e:
            hdmc.System3(*args)
        assert e.value.code == hdmc.HDMC_EINVAL
    with pytest.raises(hdmc.HDMCError) as e:
        hdmc.System3(2, [6.0] * 3, 1.0, 0.1, xyz=np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]]))
    assert e.value.code == hdmc.HDMC_EOVERLAP
    s = hdmc.System3(w.N, w.L, 1.0, 0.1)
    with pytest.raises(hdmc.HDMCError):
        s.set_move_size(0.7)
    with pytest.raises(hdmc.HDMCError):
        s.subsweep(0, 8)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_equation_of_state_carnahan_starling(prec):
    # hard-sphere fluid at phi = 0.30: Carnahan-Starling Z = (1 + p + p^2 - p^3)/(1 - p)^3
    # is within 0.05 % of simulations there
    from paper_1211_1646_gb300 import hdmc
    import torch
    phi = 0.30
    w = W.fcc3(16, phi, 0.15)
    s = hdmc.System3(w.N, w.L, 1.0, w.d, 4, 23, prec)
    s.sweep(4000)
    blocks = []
    for _ in range(12):
        for _ in range(200):
            s.sweep(5)
            s.sample()
        blocks.append(s.pressure()[0])
    torch.cuda.synchronize()
    b = np.array(blocks)
    mean, se = b.mean(), b.std(ddof=1) / math.sqrt(len(b))
    cs = (1 + phi + phi**2 - phi**3) / (1 - phi) ** 3
    print("%s: Z = %.5f +- %.5f, Carnahan-Starling %.5f" % (prec, mean, se, cs))
    assert se < 0.01
    assert abs(mean - cs) < 3 * se + 1e-3 * cs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_snapshot_resume_is_bit_identical(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.spheres_n2048_phi045()
    a = hdmc.System3(w.N, w.L, 1.0, w.d, 4, 21, prec)
    a.set_balance(False, True)
    a.sweep(7)
    a.shift()
    a.sample()
    img = a.save()
    a.sweep(9)
    a.sample()
    # a system of another seed, move and balance takes them from the image
    b = hdmc.System3(w.N, w.L, 1.0, 0.05, 4, 999, prec)
    b.load(img)
    b.sweep(9)
    b.sample()
    assert np.array_equal(a.state()[0], b.state()[0])
    assert np.array_equal(a.counters(), b.counters())
    assert np.array_equal(a.origin(), b.origin())
    pa, pb = a.pressure(), b.pressure()
    assert pa[3] == pb[3] == 2 and np.array_equal(pa[2], pb[2])
    # and both equal the oracle's straight run
    o = O.System3(w.N, w.L, 1.0, w.d, 4, 21, PREC[prec])
    o.set_balance(False, True)
    o.sweep(7)
    o.shift()
    o.sweep(9)
    assert np.array_equal(a.state()[0], o.state()[0])


def test_bad_snapshots_are_rejected_and_state_kept():
    from paper_1211_1646_gb300 import hdmc
    w = W.spheres_n2048_phi045()
    s = hdmc.System3(w.N, w.L, 1.0, w.d, 4, 22, "fp32")
    s.sweep(3)
    good = s.save()
    before = s.state()[0].copy()
    C = s.C
    cells = 256 + 256 + ((8 * 200 + 255) // 256) * 256        # header, state, histogram
    el = 4
    bad = []
    x = good.copy(); x[0] ^= 1; bad.append(x)                     # magic
    x = good.copy(); x[cells:cells + 4] = np.frombuffer(np.float32(5.0).tobytes(), np.uint8); bad.append(x)  # x >= w
    # a sphere removed: the first occupied slot 0 of some cell made empty in all three coordinates
    arr = good[cells:cells + C * 12 * el].view(np.float32).reshape(C, 12)
    k = int(np.argmax(arr[:, 0] >= 0))
    x = good.copy()
    v = x[cells:cells + C * 12 * el].view(np.float32).reshape(C, 12)
    v[k, 0] = v[k, 4] = v[k, 8] = -1.0e4
    bad.append(x)
    x = good.copy()
    v = x[cells:cells + C * 12 * el].view(np.float32).reshape(C, 12)
    v[k, 1] = 0.5 if v[k, 1] < 0 else v[k, 1]
    if v[k, 1] >= 0:                                               # slot 1 occupied after an empty slot 0
        v[k, 0] = v[k, 4] = v[k, 8] = -1.0e4
        bad.append(x)
    other = hdmc.System3(4 * 6**3, [9.0] * 3, 1.0, 0.1, 4, 1, "fp32").save()
    bad.append(other)
    for img in bad:
        with pytest.raises(hdmc.HDMCError) as e:
            s.load(img)
        assert e.value.code == hdmc.HDMC_EINVAL
        assert np.array_equal(s.state()[0], before)
    s.load(good)
    assert np.array_equal(s.state()[0], before)


def test_side_stream_matches_the_oracle():
    # a handle on a torch side stream (which does not wait for the legacy
    # default stream): creation, sweeps, a snapshot round trip, histogram
    import torch
    from paper_1211_1646_gb300 import hdmc
    w = W.spheres_n2048_phi045()
    side = torch.cuda.Stream()
    g = hdmc.System3(w.N, w.L, 1.0, w.d, 4, 31, "fp32", stream=side.cuda_stream)
    o = O.System3(w.N, w.L, 1.0, w.d, 4, 31, O.FP32)
    g.sweep(6)
    img = g.save()
    g.sweep(4)
    g.load(img)
    g.sweep(4)
    o.sweep(10)
    g.sample()
    assert np.array_equal(g.state()[0], o.state()[0])
    assert np.array_equal(g.pressure()[2], o.histogram())
