"""Parity of the CUDA library (through its C ABI) with the oracle.

Both paths are deterministic functions of (configuration, seed, sweep index):
the binary64 path must agree with the oracle's binary64 mode bit for bit,
and the binary32 path with the oracle's binary32 mode bit for bit --
positions, cell counts, slot order, trial counters, grid origin and the
contact histogram.  Sizes span several thread blocks with ragged tails;
the largest cases are the N = 1M and N = 4M workloads of the benchmark,
checked after a few sweeps against the (multi-threaded) oracle.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import pressure as P
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


def _pair(w, prec, seed=None, d=None, nsel=None, xy=None):
    from paper_1211_1646_gb300 import hdmc
    seed = w.seed if seed is None else seed
    d = w.d if d is None else d
    nsel = w.nselect if nsel is None else nsel
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, d, nsel, seed, prec, xy=xy)
    r = O.System(w.N, w.Lx, w.Ly, 1.0, d, nsel, seed, PREC[prec], xy=xy)
    return g, r


def _same(g, r, what=""):
    lg, cg = g.state()
    lr, cr = r.state()
    assert np.array_equal(cg, cr), "counts differ " + what
    bad = np.argwhere(lg != lr)
    assert bad.size == 0, "positions differ at %s %s" % (bad[:4].tolist(), what)
    assert np.array_equal(g.counters(), r.counters()), "counters differ " + what
    assert np.array_equal(g.origin(), r.origin()), "origin differs " + what


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_start_configuration(prec):
    for w in (W.n1024_phi070(), W.n65536_phi070()):
        g, r = _pair(w, prec)
        _same(g, r, "after create")
        assert np.array_equal(g.positions(), r.positions())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_n1024_200_sweeps(prec):
    w = W.n1024_phi070()
    g, r = _pair(w, prec)
    for k in range(4):
        g.sweep(50)
        r.sweep(50)
        _same(g, r, "after %d sweeps" % (50 * (k + 1)))
    assert g.info()["sweeps_done"] == 200


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_n65536_20_sweeps(prec):
    w = W.n65536_phi070()
    g, r = _pair(w, prec)
    g.sweep(20)
    r.sweep(20)
    _same(g, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_n1m_hex_phi0716(prec):
    w = W.n1m_phi0716(prec)
    g, r = _pair(w, prec)
    g.sweep(3)
    r.sweep(3)
    _same(g, r)


def test_n4m_phi0716_fp32():
    w = W.n4m(0.716, "fp32")
    g, r = _pair(w, "fp32")
    g.sweep(2)
    r.sweep(2)
    _same(g, r)


def test_n4m_phi0716_fp64():
    w = W.n4m(0.716, "fp64")
    g, r = _pair(w, "fp64")
    g.sweep(2)
    r.sweep(2)
    _same(g, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["wide", "tall", "d_max", "dilute", "dense"])
def test_geometry_and_density_extremes(prec, case):
    """Elongated boxes (shift and wrap along a long and a short axis), the
    largest legal move (just under half a cell), a dilute system (most cells
    empty) and one near close packing."""
    if case in ("wide", "tall"):
        nx, ny = (200, 8) if case == "wide" else (8, 200)
        Lx, Ly = W.hex_box(nx, ny, 0.70)
        w = W.Workload(case, nx * ny, Lx, Ly, 0.12, 4, 31, 0)
    elif case == "d_max":
        Lx, Ly = W.square_box(1024, 0.60)
        mx = 2 * int(Lx / 2)
        w = W.Workload(case, 1024, Lx, Ly, 0.499 * Lx / mx, 4, 32, 0)
    else:
        phi = 0.20 if case == "dilute" else 0.85
        nx, ny = W.hex_counts(4096)
        Lx, Ly = W.hex_box(nx, ny, phi)
        w = W.Workload(case, nx * ny, Lx, Ly, 0.15 if case == "dilute" else 0.02, 4, 33, 0)
    g, r = _pair(w, prec)
    g.sweep(70)
    r.sweep(70)
    _same(g, r, case)
    c = g.counters()
    assert c[0] == c[1] + c[2] + c[3] and c[1] > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_grid_and_nselect(prec):
    # 36 x 22 cells: set rows of 18 cells (not a multiple of 32), 11 set rows
    # (not a multiple of 4); odd n_M
    Lx, Ly = 37.3, 23.9
    N = 2 * 300
    w = W.Workload("ragged", N, Lx, Ly, 0.2, 7, 99, 0)
    g, r = _pair(w, prec)
    g.sweep(65)      # one full 64-sweep graph plus a 1-sweep graph
    r.sweep(65)
    _same(g, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiny_systems(prec):
    for N, L in ((2, 4.0), (16, 8.5)):
        w = W.Workload("tiny", N, L, L, 0.3, 4, 5, 0)
        g, r = _pair(w, prec)
        g.sweep(130)
        r.sweep(130)
        _same(g, r, "N=%d" % N)


def test_chunking_does_not_change_results():
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    a = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 3, "fp32")
    b = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 3, "fp32")
    a.sweep(130)
    for _ in range(130):
        b.sweep(1)
    assert np.array_equal(a.state()[0], b.state()[0])
    assert np.array_equal(a.counters(), b.counters())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_explicit_shift(prec):
    w = W.n1024_phi070()
    g, r = _pair(w, prec)
    g.sweep(7)
    r.sweep(7)
    for _ in range(9):
        g.shift()
        r.shift()
    _same(g, r)
    g.sweep(3)
    r.sweep(3)
    _same(g, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_many_explicit_shifts(prec):
    # 3000 shifts of a 1024-disk system: every shift direction and distance,
    # including the rare distances below 2^-9 that the binary32 path's shift
    # remaps with binary64 instructions instead of fixed point (Alg. 4).
    w = W.n1024_phi070()
    g, r = _pair(w, prec)
    g.sweep(3)
    r.sweep(3)
    for k in range(6):
        for _ in range(500):
            g.shift()
            r.shift()
        _same(g, r, "after %d shifts" % (500 * (k + 1)))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shift_edge_cases(prec):
    # Disks exactly on and one ulp inside cell edges (the ownership test of
    # Sec. 3.2 decides them), and disks with tiny local coordinates (binary32
    # values below the fixed-point range of the binary32 shift, and a
    # subnormal one), through 400 shifts and a few sweeps, bit for bit.
    from paper_1211_1646_gb300 import hdmc
    L = 17.0
    mx, my, wx, wy = O.grid(L, L)
    pts = []
    for cy in range(0, my, 2):
        for cx in range(2, mx, 2):
            base = np.array([cx * wx, cy * wy])
            for off in ([0.0, 0.0], [np.nextafter(wx, 0), np.nextafter(wy, 0)]):
                pts.append(base + off)
    tiny = [1e-30, 1e-40, 2.0**-37, 2.0**-36, 3e-12, 1e-20, 2.0**-38 + 2.0**-60, 5e-45]
    for k, v in enumerate(tiny):
        pts.append([v, (2 * k + 1) * wy])
        pts.append([2 * wx, (2 * k + 1) * wy + v])
    xy = np.array(pts)
    assert len(xy) == 128   # the library's lattice start (replaced by xy) must be legal for this N
    xy = np.where(xy >= L, xy - L, xy)
    g = hdmc.System(len(xy), L, L, 1.0, 0.1, 4, 5, prec, xy=xy)
    r = O.System(len(xy), L, L, 1.0, 0.1, 4, 5, PREC[prec], xy=xy)
    _same(g, r, "start")
    for k in range(8):
        for _ in range(50):
            g.shift()
            r.shift()
        _same(g, r, "after %d shifts" % (50 * (k + 1)))
    g.sweep(20)
    r.sweep(20)
    _same(g, r, "after sweeps")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_cell_rule(prec):
    # HDMC_CELLS_SQRT2 (Sec. 3.1 cell width just below sqrt(2) sigma): the same
    # chain as the oracle with that grid, bit for bit
    from paper_1211_1646_gb300 import hdmc
    L = W.square_box(65536, 0.708)
    g = hdmc.System(65536, L[0], L[1], 1.0, 0.1, 4, 9, prec, cells="sqrt2")
    r = O.System(65536, L[0], L[1], 1.0, 0.1, 4, 9, PREC[prec], cells=O.CELLS_SQRT2)
    assert (g.mx, g.my) == (r.mx, r.my) == (192, 192)
    _same(g, r, "start")
    g.sweep(20)
    r.sweep(20)
    _same(g, r, "after 20 sweeps")
    _, _, hist, _ = g.pressure()
    assert np.array_equal(hist, r.histogram(200, 1e-4))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nsel", [1, 7, 8])
def test_crowded_cells_any_nselect(prec, nsel):
    # Cells holding 1.3 disks or more on average (the Sec. 3.1 cells at
    # phi = 0.708) select the binary32 sub-sweep variant that keeps every
    # neighbour slot in registers; an n_M other than 4 runs its trial loop in
    # chunks of drawn directions.  A hexagonal box whose half grid (61 x 34
    # cells per set) leaves ragged blocks in both directions.
    from paper_1211_1646_gb300 import hdmc
    nx, ny = 150, 98
    Lx, Ly = W.hex_box(nx, ny, 0.708)
    N = nx * ny
    g = hdmc.System(N, Lx, Ly, 1.0, 0.12, nsel, 31, prec, cells="sqrt2")
    r = O.System(N, Lx, Ly, 1.0, 0.12, nsel, 31, PREC[prec], cells=O.CELLS_SQRT2)
    assert (g.mx, g.my) == (r.mx, r.my) == (122, 68)
    assert 10 * N >= 13 * g.mx * g.my   # the crowded-cell rule of the library
    _same(g, r, "start")
    g.sweep(10)
    r.sweep(10)
    _same(g, r, "after 10 sweeps")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_contact_histogram_and_pressure(prec):
    w = W.n65536_phi070()
    g, r = _pair(w, prec)
    hr = np.zeros(200, dtype=np.uint64)
    for k in range(3):
        g.sweep(10)
        r.sweep(10)
        g.sample()
        hr += r.histogram()
    bp, g0, hist, ns = g.pressure()
    assert ns == 3
    assert np.array_equal(hist, hr)
    bp_ref, g0_ref, _ = P.pressure(hr, 3, w.N, w.Lx * w.Ly)
    assert abs(g0 - g0_ref) < 1e-9 * abs(g0_ref)
    assert abs(bp - bp_ref) < 1e-9 * abs(bp_ref)
    # the accumulator was cleared: the next call samples the current state
    bp2, _, hist2, ns2 = g.pressure()
    assert ns2 == 1 and np.array_equal(hist2, r.histogram())


def test_histogram_at_1m():
    w = W.n1m_phi0716("fp32")
    g, r = _pair(w, "fp32")
    g.sweep(2)
    r.sweep(2)
    _, _, hist, _ = g.pressure()
    assert np.array_equal(hist, r.histogram())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_set_positions_and_errors(prec):
    from paper_1211_1646_gb300 import hdmc
    L = 20.0
    w = W.Workload("rsa", 40, L, L, 0.25, 4, 8, 0)
    rng = np.random.default_rng(5)
    pts = []
    while len(pts) < 40:
        p = rng.uniform(0, L, 2)
        if all(math.hypot(*((p - q) - L * np.round((p - q) / L))) > 1.05 for q in pts):
            pts.append(p)
    xy = np.array(pts)
    g, r = _pair(w, prec, xy=xy)
    _same(g, r, "after set_positions")
    g.sweep(40)
    r.sweep(40)
    _same(g, r)
    bad = xy.copy()
    bad[1] = bad[0] + [0.5, 0.0]
    bad[1] %= L
    with pytest.raises(hdmc.HDMCError) as e:
        hdmc.hdmc_set_positions(g.h, bad)
    assert e.value.code == hdmc.HDMC_EOVERLAP
    _same(g, r, "state kept after a rejected set_positions")
    with pytest.raises(hdmc.HDMCError) as e:
        hdmc.System(40, L, L, 1.0, 0.9, 4, 1, prec)
    assert e.value.code == hdmc.HDMC_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_is_bit_identical(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    a = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 12, prec)
    a.sweep(100)
    loc, cnt = a.state()
    info = a.info()
    b = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 12, prec)
    b.set_state(loc, cnt, info["origin"], info["sweeps_done"], info["shifts_done"])
    a.sweep(100)
    b.sweep(100)
    assert np.array_equal(a.state()[0], b.state()[0])
    assert np.array_equal(a.positions(), b.positions())


def test_torch_side_stream():
    import torch
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 1, "fp64")
        g.sweep(30)
    r = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 1, O.FP64)
    r.sweep(30)
    _same(g, r)


def test_invariants_on_gpu_fp32_long_run():
    # 2000 sweeps at phi = 0.716: particle count, n <= 4, containment, no overlap
    from paper_1211_1646_gb300 import hdmc
    w = W.n65536_phi070()
    Lx, Ly = W.hex_box(256, 256, 0.716)
    g = hdmc.System(65536, Lx, Ly, 1.0, 0.08, 4, 77, "fp32")
    g.sweep(2000)
    loc, cnt = g.state()
    assert int(cnt.sum()) == 65536 and cnt.max() <= 4
    occ = np.arange(4)[None, :] < cnt[:, None]
    wx32 = float(np.float32(g.wx))
    wy32 = float(np.float32(g.wy))
    assert np.all((loc[..., 0][occ] >= 0) & (loc[..., 0][occ] < wx32))
    assert np.all((loc[..., 1][occ] >= 0) & (loc[..., 1][occ] < wy32))
    from scipy.spatial import cKDTree
    bx, by = g.box()
    xy = g.positions()
    assert xy.min() >= 0 and xy[:, 0].max() < bx and xy[:, 1].max() < by
    pairs = cKDTree(xy, boxsize=[bx, by]).query_pairs(1.0 - 1e-6)
    assert len(pairs) == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nsel", [1, 8, 12, 20])
def test_trials_per_cell(prec, nsel):
    # n_M = 1, n_M = 8 (a binary32 kernel with n_M fixed, its directions
    # drawn in one pass) and n_M above the 8 directions drawn ahead per
    # block of work
    w = W.n1024_phi070()
    g, r = _pair(w, prec, nsel=nsel, seed=4)
    g.sweep(25)
    r.sweep(25)
    _same(g, r)
