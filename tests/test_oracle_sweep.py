"""Pins for the oracle's sweep, shift and pressure estimator (CPU only).

What fixes the expected values here:
  - invariants the paper states (no overlap, particle count conserved by the
    shift, moves never leave their cell, n <= 4 for w < sqrt(2) sigma);
  - brute force over all pairs in global coordinates;
  - the stationary distribution that detailed balance implies: uniform over
    legal configurations (two disks on a torus, and tiny systems compared
    with independent rejection sampling);
  - the paper's estimator calibration (model distribution, Sec. 4) and an
    ideal gas (g = 1);
  - the low-density virial series of hard disks (textbook closed forms).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from oracle import pressure as P
from paper_1211_1646_gb300 import workloads as W

from golden import keyvals


def _global_ok(sys_, rmin_factor):
    Lx, Ly = sys_.box()
    xy = sys_.positions()
    return O.close_pairs(xy, Lx, Ly, sys_.sigma * rmin_factor)


def test_grid_rule():
    # Eq. 1 needs an even number of cells per axis on a periodic box;
    # cells are the smallest such width >= sigma.
    w1 = W.n1024_phi070()
    mx, my, wx, wy = O.grid(w1.Lx, w1.Ly)
    assert (mx, my) == (32, 32) and abs(wx - 1.0592437756635953) < 1e-12
    w2 = W.n65536_phi070()
    mx, my, wx, wy = O.grid(w2.Lx, w2.Ly)
    assert (mx, my) == (270, 270) and 1.0043 < wx < 1.0044
    w3 = W.n1m_phi0716()
    mx, my, wx, wy = O.grid(w3.Lx, w3.Ly)
    assert (mx, my) == (1152, 998) and wx >= 1.0 and wy >= 1.0
    with pytest.raises(ValueError):
        O.grid(3.9, 10.0)          # fewer than 4 cells
    with pytest.raises(ValueError):
        O.grid(5.8, 10.0)          # 4 cells of 1.45 sigma > sqrt(2) sigma (Fig. 3)


def test_cell_rule_fig3_bound():
    g = keyvals("cell_rule_fig3.txt")
    # five centres at the corners and the middle of a square of edge w are
    # pairwise >= sigma apart exactly when w >= sqrt(2) sigma
    w5 = g["w5_over_sigma"]
    pts = lambda w: np.array([[0, 0], [w, 0], [0, w], [w, w], [w / 2, w / 2]])
    dmin = lambda p: min(np.hypot(*(p[i] - p[j])) for i in range(5) for j in range(i + 1, 5))
    assert dmin(pts(w5)) >= 1.0 - 1e-12
    assert dmin(pts(w5 * (1 - 1e-6))) < 1.0


def test_lattice_start():
    w = W.n1024_phi070()
    assert O.lattice_shape(w.N, w.Lx, w.Ly) == (32, 32)
    w3 = W.n1m_phi0716()
    assert O.lattice_shape(w3.N, w3.Lx, w3.Ly) == (1024, 1024)
    xy = O.lattice_positions(w.N, w.Lx, w.Ly, 1.0, 1)
    assert np.all((xy >= 0) & (xy < [w.Lx, w.Ly]))
    assert O.close_pairs(xy, w.Lx, w.Ly, 1.0) == 0
    # jitter is within 0.01 sigma of the ideal sites
    nx, ny = 32, 32
    j, i = np.divmod(np.arange(w.N), nx)
    ideal = np.stack([(i + 0.5 + 0.5 * (j % 2)) * w.Lx / nx, (j + 0.5) * w.Ly / ny], axis=1)
    dd = xy - ideal
    dd -= np.array([w.Lx, w.Ly]) * np.round(dd / [w.Lx, w.Ly])
    r = np.hypot(dd[:, 0], dd[:, 1])
    assert r.max() < 0.01 and r.max() > 0.005


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_sweep_invariants(prec):
    w = W.n1024_phi070()
    s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, prec)
    tol = 1e-9 if prec == O.FP64 else 1e-6
    for k in range(40):
        s.sweep(1)
        loc, cnt = s.state()
        assert int(cnt.sum()) == w.N                       # shift conserves particles
        assert cnt.max() <= 4                              # n_max = 4 (Fig. 3)
        occ = np.arange(4)[None, :] < cnt[:, None]
        wxs = s.wx if prec == O.FP64 else float(np.float32(s.wx))
        lx, ly = loc[..., 0][occ], loc[..., 1][occ]
        assert np.all((lx >= 0) & (lx < wxs) & (ly >= 0) & (ly < wxs))   # inside own cell
        assert np.all(loc[~occ] == O.EMPTY_SLOT)
        if k % 8 == 0:
            assert _global_ok(s, 1 - tol) == 0             # no overlap anywhere
            assert s.local_overlaps() == 0
    c = s.counters()
    assert c[0] == c[1] + c[2] + c[3] and c[1] > 0 and c[2] > 0 and c[3] > 0


def test_trial_count_is_nselect_per_occupied_cell():
    w = W.n1024_phi070()
    s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 3, w.seed, O.FP64)
    s.sweep(5)
    _, cnt = s.state()
    cnt = cnt.reshape(s.my, s.mx)
    before = s.counters()
    s.subsweep(77, 2)   # set c: even x, odd y (Eq. 1)
    after = s.counters()
    occupied = int((cnt[1::2, 0::2] > 0).sum())
    assert int(after[0] - before[0]) == 3 * occupied


def test_shift_is_a_relabelling():
    w = W.n1024_phi070()
    for prec in (O.FP64, O.FP32):
        s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 3, prec)
        s.sweep(10)
        Lx, Ly = s.box()
        a = s.positions()
        o0 = s.origin()
        for _ in range(25):
            s.shift()
        b = s.positions()
        assert not np.array_equal(s.origin(), o0)
        key = lambda xy: xy[np.lexsort((xy[:, 1], xy[:, 0]))]
        # same multiset of positions modulo the box: binary64 mode only rounds
        # O + cell*w + local; binary32 mode also rounds each remapped offset to
        # binary32 (at most half an ulp of w per shift)
        d = key(a) - key(b)
        d -= np.array([Lx, Ly]) * np.round(d / [Lx, Ly])
        tol = 1e-11 if prec == O.FP64 else 25 * 2.0**-24 * 1.06
        assert np.abs(d).max() < tol


def test_binary32_shift_rounds_each_coordinate_once():
    # Alg. 4 translates every disk by -f*ds.  In the binary32 mode the
    # translation, the ownership test and the re-expression in the new cell
    # are binary64, and only the stored result is rounded to binary32: each
    # shift moves a disk's global position by at most half an ulp of its new
    # binary32 local coordinate (plus the binary64 rounding of O + cell*w +
    # local).  A binary32 remap rounds a migrant twice (x - ds, then + w) and
    # breaks this bound.
    w = W.n1024_phi070()
    s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 3, O.FP32)
    s.sweep(10)
    Lx, Ly = s.box()
    worst = 0.0
    for _ in range(60):
        a = s.positions()
        s.shift()
        b = s.positions()
        loc, cnt = s.state()
        bl = loc[np.arange(4)[None, :] < cnt[:, None]]       # canonical order, like positions()
        ia, ib = np.lexsort((a[:, 1], a[:, 0])), np.lexsort((b[:, 1], b[:, 0]))
        d = a[ia] - b[ib]
        d -= np.array([Lx, Ly]) * np.round(d / [Lx, Ly])
        half = 0.5 * np.spacing(bl[ib].astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(d) <= half + 1e-12)
        worst = max(worst, float((np.abs(d) / (half + 1e-300)).max()))
    assert worst > 0.5   # the bound is approached, so the test has teeth


def test_shift_conserves_particles_on_cell_edges():
    # disks sitting exactly on, or one ulp inside, cell edges
    L = 12.0
    mx, my, wx, wy = O.grid(L, L)
    pts = []
    for cy in range(0, my, 2):
        for cx in range(0, mx, 2):
            base = np.array([cx * wx, cy * wy])
            for off in ([0.0, 0.0], [np.nextafter(wx, 0), np.nextafter(wy, 0)]):
                pts.append(base + off)
    xy = np.array(pts)
    xy = np.where(xy >= L, xy - L, xy)
    for prec in (O.FP64, O.FP32):
        s = O.System(len(xy), L, L, 1.0, 0.1, 4, 5, prec, xy=xy)
        for k in range(400):
            s.shift()
            loc, cnt = s.state()
            assert int(cnt.sum()) == len(xy)
        assert s.local_overlaps() == 0


def test_openmp_thread_count_does_not_change_results():
    w = W.n1024_phi070()
    res = []
    for nt in (1, 4):
        O.set_threads(nt)
        s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 9, O.FP64)
        s.sweep(20)
        res.append((s.state()[0].copy(), s.counters().copy()))
    O.set_threads(1)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_split_runs_are_identical():
    w = W.n1024_phi070()
    a = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 21, O.FP32)
    b = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 21, O.FP32)
    a.sweep(30)
    for _ in range(3):
        b.sweep(10)
    assert np.array_equal(a.state()[0], b.state()[0])
    assert np.array_equal(a.counters(), b.counters())


def test_errors():
    L = 10.0
    with pytest.raises(O.OracleError) as e:
        O.System(2, L, L, 1.0, 0.1, 4, 1, O.FP64, xy=np.array([[1.0, 1.0], [1.5, 1.0]]))
    assert e.value.code == O.EOVERLAP
    with pytest.raises(O.OracleError) as e:
        O.System(2, L, L, 1.0, 0.7, 4, 1, O.FP64)   # d >= w/2
    assert e.value.code == O.EINVAL
    with pytest.raises(O.OracleError) as e:
        # five centres in one 1.25-sigma cell must overflow it
        xy = np.array([[0.1, 0.1], [0.2, 0.2], [0.3, 0.3], [0.4, 0.4], [0.5, 0.5]])
        O.System(5, L, L, 1.0, 0.1, 4, 1, O.FP64, xy=xy)
    assert e.value.code == O.EOVERFLOW


def _min_image(d, L):
    return d - L * np.round(d / L)


# Smallest separation the binary32 chain may produce: its overlap test is
# fma(dx, dx, fma(dy, dy, -sigma^2)) < 0 on binary32 cell-local coordinates,
# whose rounding (a few ulp of sigma^2 = 1) admits pairs a hair inside sigma.
R_MIN = {O.FP64: 1.0 - 1e-12, O.FP32: 1.0 - 1e-6}


@pytest.mark.parametrize("strips", [0, 2])
@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_two_disks_sample_the_uniform_distribution(prec, strips):
    # Detailed balance (Sec. 2.3) makes the uniform measure on legal
    # configurations stationary: the separation of two disks on a 4x4 torus
    # is uniform over the square [-2,2)^2 minus the disk |r| < sigma.  Both
    # arithmetic modes of the oracle must sample it.
    L = 4.0
    # strips = 2: the spatial decomposition of Sec. 6, rows 0 and 2 of the
    # 4-row grid make no moves during the sub-sweeps; the grid shift moves
    # the frozen rows over the disks, and the chain samples the same measure
    s = O.System(2, L, L, 1.0, 0.45, 4, 2024, prec, xy=np.array([[0.5, 0.5], [2.5, 2.5]]))
    s.set_strips(strips)
    assert s.box() == (L, L)
    s.sweep(200)
    seps = []
    for _ in range(40000):
        s.sweep(8)
        xy = s.positions()
        seps.append([_min_image(xy[1, 0] - xy[0, 0], L), _min_image(xy[1, 1] - xy[0, 1], L)])
    seps = np.array(seps)
    r = np.hypot(seps[:, 0], seps[:, 1])
    assert r.min() >= R_MIN[prec]
    inside = r < 2.0
    p_in = 3 * math.pi / (16 - math.pi)
    # correlated samples: allow for an effective sample size of a quarter
    n_eff = len(r) / 4
    assert abs(inside.mean() - p_in) < 4 * math.sqrt(p_in * (1 - p_in) / n_eff)
    ri = r[inside]
    assert stats.kstest((ri**2 - 1) / 3, "uniform").statistic < 1.6 / math.sqrt(len(ri) / 4)
    # disks carry no labels (positions come back in cell order), so the
    # separation is that of an unordered pair: fold the angle onto [0, pi)
    th = np.mod(np.arctan2(seps[:, 1], seps[:, 0])[inside], math.pi) / math.pi
    assert stats.kstest(th, "uniform").statistic < 1.6 / math.sqrt(len(th) / 4)
    # the 2-d density of the separation is flat on the square minus the disk
    seps = np.concatenate([seps, -seps])
    r = np.concatenate([r, r])
    grid = np.floor((seps + 2) / 0.5).astype(int).clip(0, 7)
    far = r > 1.5 ** 0.5 * 1.5   # cells wholly outside the excluded disk
    tab = np.bincount((grid[:, 0] * 8 + grid[:, 1])[far], minlength=64)
    cells = [(i, j) for i in range(8) for j in range(8)
             if min(math.hypot(-2 + 0.5 * a, -2 + 0.5 * b) for a in (i, i + 1) for b in (j, j + 1)) > 1.85]
    sel = np.array([tab[i * 8 + j] for i, j in cells])
    assert sel.min() > 0.8 * sel.mean() and sel.max() < 1.2 * sel.mean()


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_two_disk_pin_detects_moves_that_leave_the_cell(prec):
    # Sec. 2.4 item 1: letting a disk leave its cell during a sub-sweep
    # breaks detailed balance.  The oracle's negative-control switch does
    # exactly that (the disk moves into the neighbouring cell when it
    # overlaps nothing there); the two-disk pin above must reject the chain,
    # in both arithmetic modes.
    L = 4.0
    s = O.System(2, L, L, 1.0, 0.45, 4, 2024, prec, xy=np.array([[0.5, 0.5], [2.5, 2.5]]))
    s.set_allow_leave(True)
    s.sweep(200)
    r = []
    for _ in range(80000):
        s.sweep(8)
        xy = s.positions()
        r.append(math.hypot(_min_image(xy[1, 0] - xy[0, 0], L), _min_image(xy[1, 1] - xy[0, 1], L)))
    r = np.array(r)
    assert r.min() >= R_MIN[prec]                       # still no overlap
    ri = r[r < 2.0]
    crit = 1.6 / math.sqrt(len(ri) / 4)
    assert stats.kstest((ri**2 - 1) / 3, "uniform").statistic > crit
    # the separations near contact are under-sampled
    near = np.mean(ri < 1.2) / ((1.2**2 - 1) / 3)
    assert near < 0.93
    c = s.counters()
    assert c[2] == 0 and c[1] > 0.9 * c[0]              # no move is rejected for leaving


@pytest.mark.parametrize("strips", [0, 2])
@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_tiny_system_matches_rejection_sampling(prec, strips):
    # 4 disks on a 4.4 x 4.4 torus: pair-distance distribution of the Markov
    # chain equals that of independent uniform legal configurations.  With
    # cells of width 1.1, two disks share a cell often enough that a wrong
    # own-cell exclusion or visit order shows up here.
    L = 4.4
    rng = np.random.default_rng(8)
    ref = []
    while len(ref) < 30000:
        xy = rng.uniform(0, L, (4, 2))
        ds = [math.hypot(*_min_image(xy[i] - xy[j], L)) for i in range(4) for j in range(i + 1, 4)]
        if min(ds) >= 1.0:
            ref.append(min(ds))
    start = np.array([[0.5, 0.5], [2.7, 0.5], [0.5, 2.7], [2.7, 2.7]])
    s = O.System(4, L, L, 1.0, 0.4, 4, 77, prec, xy=start)
    s.set_strips(strips)   # 2: inactive bands on rows 0 and 2 (Sec. 6)
    Lx, Ly = s.box()   # binary32 mode: 4 x float(1.1), a hair above 4.4
    s.sweep(200)
    mc = []
    shared = 0
    for _ in range(15000):
        s.sweep(6)
        xy = s.positions()
        ds = [math.hypot(_min_image(xy[i, 0] - xy[j, 0], Lx), _min_image(xy[i, 1] - xy[j, 1], Ly))
              for i in range(4) for j in range(i + 1, 4)]
        mc.append(min(ds))
        shared += int((s.state()[1] > 1).any())
    assert min(mc) >= R_MIN[prec]
    assert shared > 300   # configurations with two disks in one cell are sampled (about 3 %)
    res = stats.ks_2samp(np.array(ref), np.array(mc))
    n_eff = 15000 / 3
    crit = 1.95 * math.sqrt((1 / n_eff) + (1 / len(ref)))
    assert res.statistic < crit


def test_histogram_equals_brute_force():
    w = W.n1024_phi070()
    for prec in (O.FP64, O.FP32):
        s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 4, prec)
        s.sweep(60)
        h = s.histogram(200, 1e-4)
        Lx, Ly = s.box()
        hb = O.bruteforce_histogram(s.positions(), Lx, Ly, 1.0, 200, 1e-4)
        assert h.sum() > 100
        assert np.array_equal(h, hb)
        # ordered pairs: every pair counted from both ends
        assert h.sum() % 2 == 0


def _pair_histogram_kdtree(xy, L, sigma, nbins, dr):
    """Ordered-pair distance histogram with scipy's periodic k-d tree."""
    from scipy.spatial import cKDTree
    t = cKDTree(xy, boxsize=L)
    pairs = t.query_pairs(sigma + nbins * dr, output_type="ndarray")
    d = xy[pairs[:, 0]] - xy[pairs[:, 1]]
    d -= L * np.round(d / L)
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    e = sigma + np.arange(nbins + 1) * dr
    E = e * e
    keep = (r2 >= E[0]) & (r2 < E[-1])
    b = np.searchsorted(E, r2[keep], side="right") - 1
    return 2 * np.bincount(b, minlength=nbins)


def test_ideal_gas_contact_value_is_one():
    # Eq. gR with ordered pairs: uniform independent points give g = 1.
    Lx = Ly = 120.0
    N = 20000
    nconf = 10
    hist = np.zeros(200, dtype=np.float64)
    for k in range(nconf):
        xy = W.uniform_points(N, Lx, Ly, 100 + k)
        hist += _pair_histogram_kdtree(xy, Lx, 1.0, 200, 1e-4)
    R, g = P.g_of_r(hist, nconf, N, Lx * Ly, 1.0, 1e-4)
    assert abs(g.mean() - 1) < 4 / math.sqrt(hist.sum() / 2)
    g0 = P.contact_value(R, g, 1.0, 0.02)
    assert abs(g0 - 1) < 4 * 6 / math.sqrt(hist.sum() / 2)


def test_squared_bin_edges():
    # bin b covers [sigma + b dr, sigma + (b+1) dr): its squared edges are
    # increasing and within rounding of the exact squares
    E = O.squared_bin_edges(1.0, 1e-4, 200)
    exact = (1.0 + 1e-4 * np.arange(201)) ** 2
    assert np.all(np.diff(E) > 0) and np.allclose(E, exact, rtol=1e-15, atol=0)


def test_bruteforce_histogram_matches_kdtree():
    L = 30.0
    xy = W.uniform_points(900, L, L, 5)
    a = O.bruteforce_histogram(xy, L, L, 1.0, 200, 1e-4)
    b = _pair_histogram_kdtree(xy, L, 1.0, 200, 1e-4)
    assert a.sum() > 0 and np.array_equal(a, b)


def _model_counts(amp, rate, sigma, dr, nbins):
    r = P.bin_edges(sigma, dr, nbins)
    # n(r) = 2 pi r g_m(r), g_m(r) = amp exp(-rate (r - sigma)), integrated over each bin
    F = lambda x: -amp * np.exp(-rate * (x - sigma)) * (x / rate + 1 / rate**2)
    return 2 * np.pi * (F(r[1:]) - F(r[:-1]))


def test_estimator_calibration_on_model_distribution():
    g = keyvals("estimator_sec4.txt")
    amp, rate = g["model_amplitude"], g["model_rate"]
    n = _model_counts(amp, rate, 1.0, g["dr"], 200)
    R, gr = P.g_of_r(n, 1, 1, 1.0, 1.0, g["dr"])
    g0 = P.contact_value(R, gr, 1.0, g["c"], g["degree"])
    assert abs(g0 / amp - 1) < g["max_relative_bias"]
    # a lower degree does not meet the paper's bias bound
    assert abs(P.contact_value(R, gr, 1.0, g["c"], 3) / amp - 1) > g["max_relative_bias"]
    # a second least-squares routine agrees
    alt = np.polyval(np.polyfit((R - 1.0) / g["c"], gr, g["degree"]), 0.0)
    assert abs(alt - g0) < 1e-9 * amp


def test_pressure_formula_closed_form():
    # Eq. P at g(sigma+) = 1: beta P / rho = 1 + B2 rho with B2 = pi sigma^2 / 2
    r = P.bin_edges(1.0, 1e-4, 200)
    n = np.pi * (r[1:] ** 2 - r[:-1] ** 2)          # n(r) = 2 pi r, i.e. g = 1
    N, area = 1, 1.0
    bp, g0, pstar = P.pressure(n, 1, N, area)
    assert abs(g0 - 1) < 1e-6
    rho = N / area
    assert abs(bp - (1 + math.pi / 2 * rho)) < 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_low_density_virial_series(prec):
    # beta P / rho = 1 + B2 rho + B3 rho^2 + B4 rho^3 + ... for hard disks:
    # B2 = pi sigma^2/2, B3/B2^2 = 4/3 - sqrt(3)/pi, B4/B2^3 = 2 - 9 sqrt(3)/(2 pi) + 10/pi^2.
    phi = 0.10
    N = 1024
    Lx, Ly = W.square_box(N, phi)
    rho = N / (Lx * Ly)
    B2 = math.pi / 2
    B3 = B2**2 * (4 / 3 - math.sqrt(3) / math.pi)
    B4 = B2**3 * (2 - 9 * math.sqrt(3) / (2 * math.pi) + 10 / math.pi**2)
    B5 = B2**4 * 0.3335
    series = 1 + B2 * rho + B3 * rho**2 + B4 * rho**3 + B5 * rho**4
    s = O.System(N, Lx, Ly, 1.0, 0.45, 4, 31, prec)
    area = s.box()[0] * s.box()[1]
    s.sweep(300)
    blocks = []
    for b in range(20):
        h = np.zeros(200)
        for k in range(250):
            s.sweep(2)
            h += s.histogram(200, 1e-4)
        blocks.append(P.pressure(h, 250, N, area)[0])
    blocks = np.array(blocks)
    mean, se = blocks.mean(), blocks.std(ddof=1) / math.sqrt(len(blocks))
    assert abs(mean - series) < 3 * se + 1e-3, (mean, se, series)
    # the second-order term alone is resolved
    assert abs(mean - (1 + B2 * rho)) > 3 * se


def test_inactive_bands_make_no_moves():
    # Sec. 6 decomposition: strip k starts at row 2 floor(k my / (2R)); that
    # row makes no trial moves during the sub-sweeps, every other cell makes
    # n_M (trials = n_M x occupied cells off the band rows), and the band
    # rows' disks still move with the grid shift.
    w = W.n1024_phi070()
    for prec in (O.FP64, O.FP32):
        for R in (1, 3, 16):
            s = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 9, prec)
            s.set_strips(R)
            rows = s.strip_rows(R)
            assert rows[0][0] == 0 and rows[-1][1] == s.my
            assert all(b - a >= 2 and a % 2 == 0 for a, b in rows)
            band = [a for a, _ in rows]
            for sweep in range(3):
                loc, cnt = s.state()
                before = [s.get_row(r)[0].copy() for r in band]
                occ = cnt.reshape(s.my, s.mx)
                active = int((occ > 0).sum() - sum((occ[r] > 0).sum() for r in band))
                c0 = s.counters().copy()
                for Q in range(4):
                    s.subsweep(sweep, Q)
                assert int(s.counters()[0] - c0[0]) == 4 * active
                for r, b in zip(band, before):
                    assert np.array_equal(s.get_row(r)[0], b)
            s.sweep(20)
            assert s.local_overlaps() == 0 and int(s.state()[1].sum()) == w.N
    with pytest.raises(ValueError):
        O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 9, O.FP64).set_strips(17)   # my = 32 < 2 x 17


def test_paper_cell_rule():
    # Sec. 3.1: m = floor(L / (sqrt(2) sigma)) rounded up, here to the next
    # even integer (the checkerboard on a periodic box): the widest cells
    # below sqrt(2) sigma, which still hold at most four centres (Fig. 3).
    for L in (30.0, 100.0, 269.63, 1152.45):
        mx, my, wx, wy = O.grid(L, L, 1.0, O.CELLS_SQRT2)
        assert mx % 2 == 0 and 1.0 <= wx < math.sqrt(2.0)
        assert L / (mx - 2) >= math.sqrt(2.0)            # two fewer cells would be too wide
        assert O.grid(L, L)[0] >= mx
    w = W.square_box(65536, 0.708)
    assert O.grid(w[0], w[1], 1.0, O.CELLS_SQRT2)[0] == 192   # N = 256^2, phi = 0.708
    w = W.square_box(16384, 0.708)
    for prec in (O.FP64, O.FP32):
        s = O.System(16384, w[0], w[1], 1.0, 0.1, 4, 2, prec, cells=O.CELLS_SQRT2)
        s.sweep(40)
        _, cnt = s.state()
        Lx, Ly = s.box()
        # binary32 positions re-rounded by the shift may sit a hair inside contact
        assert O.close_pairs(s.positions(), Lx, Ly, R_MIN[prec]) == 0
        assert int(cnt.sum()) == 16384 and cnt.max() <= 4
        assert cnt.mean() > 1.7                           # about 1.8 disks per cell (0.9 with the default rule)

