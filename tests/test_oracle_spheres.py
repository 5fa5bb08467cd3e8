"""Pins for the oracle's three-dimensional (hard-sphere) form of the method
(CPU only).  The paper states the 3-d case in words (eight checkerboard
sets, Sec. 2.1 and 2.2; Sec. 6); what fixes the expected values here:
  - geometry: the cell-occupancy bound behind eight slots per cell;
  - invariants: no overlap, sphere count conserved by the shift, moves stay
    in their cell, the shift only relabels;
  - brute force over all pairs and periodic images in global coordinates,
    and a periodic k-d tree;
  - the stationary distribution that detailed balance implies: uniform over
    legal configurations (two spheres on a torus; four spheres compared with
    independent rejection sampling);
  - the random draws: exact bijection of the shuffle decode, uniform
    permutations, directions uniform in the unit ball;
  - the pressure estimator in three dimensions: an ideal gas (g = 1), the
    closed form at g = 1, a model distribution, and the hard-sphere virial
    series at low density (textbook coefficients).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from oracle import pressure as P
from paper_1211_1646_gb300 import workloads as W

from golden import keyvals


@pytest.fixture(scope="module", autouse=True)
def built():
    from oracle import build
    build.build()


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_grid_rule_3d():
    m, w = O.grid3([20.0, 20.0, 20.0])
    assert list(m) == [20, 20, 20] and np.all(w == 1.0)
    m, w = O.grid3([13.36, 26.7, 10.9])
    assert list(m) == [12, 26, 10]
    assert np.allclose(w, [13.36 / 12, 26.7 / 26, 10.9 / 10])
    with pytest.raises(ValueError):
        O.grid3([3.9, 10.0, 10.0])          # fewer than 4 cells on an axis
    with pytest.raises(ValueError):
        O.grid3([13.9, 13.9, 13.9])         # 12 cells of 1.158: 3 w^2 >= 4 sigma^2
    # one long axis may take the slack the other two leave
    m, w = O.grid3([10.0, 10.0, 13.9])
    assert (w**2).sum() < 4.0


def test_eight_slots_bound():
    # the eight corners of a cube of edge w are pairwise >= sigma apart iff
    # w >= sigma; a ninth centre (the body centre) fits iff w >= 2 sigma/sqrt(3),
    # which the grid rule excludes (sum of w^2 < 4 sigma^2 keeps each of the
    # eight half-size boxes of a cell below one diameter across)
    def dmin(p):
        return min(np.linalg.norm(p[i] - p[j]) for i in range(len(p)) for j in range(i + 1, len(p)))
    corners = lambda w: np.array(list(itertools.product([0.0, w], repeat=3)))
    nine = lambda w: np.vstack([corners(w), [[w / 2] * 3]])
    assert dmin(corners(1.0)) >= 1.0 - 1e-12 and dmin(corners(0.999)) < 1.0
    w9 = 2.0 / math.sqrt(3.0)
    assert dmin(nine(w9)) >= 1.0 - 1e-12
    assert dmin(nine(w9 * (1 - 1e-6))) < 1.0
    # and the oracle accepts a cell holding eight spheres
    w = 1.1
    xyz = 0.01 + np.array(list(itertools.product([0.0, 1.05], repeat=3)))
    s = O.System3(8, [4 * w] * 3, 1.0, 0.1, 8, 3, O.FP64, xyz=xyz)
    loc, cnt = s.state()
    assert cnt.max() == 8 and cnt.sum() == 8
    s.sweep(20)
    assert s.state()[1].sum() == 8 and O.close_pairs3(s.positions(), s.box(), 1.0) == 0


def test_fcc_start():
    w = W.spheres_n2048_phi045()
    xyz = O.lattice3_positions(w.N, w.L, 1.0, 7)
    q = 8
    a = np.array(w.L) / q
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    ideal = np.array([(np.array([i, j, k]) + b + 0.25) * a
                      for k in range(q) for j in range(q) for i in range(q) for b in basis])
    dev = np.linalg.norm(_min_image(xyz - ideal, np.array(w.L)), axis=1)
    assert dev.max() <= 0.01 + 1e-12 and dev.min() > 0
    assert np.all(xyz >= 0) and np.all(xyz < np.array(w.L))
    s = O.System3(w.N, w.L, 1.0, w.d, 4, 7, O.FP64)
    assert s.local_overlaps() == 0
    nn = a[0] / math.sqrt(2)                        # fcc nearest-neighbour distance
    assert O.close_pairs3(s.positions(), w.L, nn - 0.021) == 0
    assert O.close_pairs3(s.positions(), w.L, nn + 0.021) == 6 * w.N   # 12 neighbours each
    with pytest.raises(ValueError):
        O.lattice3_positions(2000, w.L, 1.0, 7)    # not 4 q^3


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_sweep_invariants_3d(prec):
    w = W.spheres_n2048_phi045()
    s = O.System3(w.N, w.L, 1.0, w.d, 4, 11, prec)
    s.sweep(25)
    loc, cnt = s.state()
    assert cnt.sum() == w.N and cnt.max() <= 8
    wl = s.w if prec == O.FP64 else s.w.astype(np.float32).astype(np.float64)
    occ = np.arange(8)[None, :] < cnt[:, None]
    for a in range(3):
        v = loc[:, :, a][occ]
        assert v.min() >= 0 and v.max() < wl[a]
    assert np.all(loc[~occ] == O.EMPTY_SLOT)
    assert s.local_overlaps() == 0
    rmin = 1.0 if prec == O.FP64 else 1.0 - 1e-6
    assert O.close_pairs3(s.positions(), s.box(), rmin) == 0
    c = s.counters()
    assert c[0] == c[1] + c[2] + c[3] and c[0] % 4 == 0
    assert 0.2 < c[1] / c[0] < 0.8


def test_trial_count_and_moves_stay_in_cell():
    w = W.spheres_n2048_phi045()
    s = O.System3(w.N, w.L, 1.0, w.d, 5, 12, O.FP64)
    s.sweep(3)
    _, cnt0 = s.state()
    m = s.m
    c0 = s.counters()
    for Q in range(8):
        s.subsweep(1000 + Q, Q)
    _, cnt1 = s.state()
    assert np.array_equal(cnt0, cnt1)               # a sub-sweep never moves a sphere to another cell
    cz, cy, cx = np.unravel_index(np.arange(s.C), (m[2], m[1], m[0]))
    assert int((s.counters() - c0)[0]) == 5 * int((cnt0 > 0).sum())
    Q = (cx & 1) + 2 * (cy & 1) + 4 * (cz & 1)
    s2 = O.System3(w.N, w.L, 1.0, w.d, 5, 12, O.FP64)
    s2.sweep(3)
    a0 = s2.counters()
    s2.subsweep(77, 5)
    assert int((s2.counters() - a0)[0]) == 5 * int(((cnt0 > 0) & (Q == 5)).sum())


def test_shift_is_a_relabelling_3d():
    w = W.spheres_n2048_phi045()
    s = O.System3(w.N, w.L, 1.0, w.d, 4, 13, O.FP64)
    s.sweep(5)
    L = np.array(w.L)
    for _ in range(12):
        before = s.positions()
        o0 = s.origin()
        s.shift()
        after = s.positions()
        do = s.origin() - o0
        assert np.count_nonzero(do) == 1 and np.all(np.abs(do) <= s.w / 2)
        key = lambda p: np.lexsort((p[:, 2], p[:, 1], p[:, 0]))
        # global positions are unchanged (up to the rounding of re-expressing
        # a migrant in its new cell's frame)
        A, B = before[key(before)], after[key(after)]
        assert np.abs(_min_image(A - B, L)).max() < 1e-9


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_shift_conserves_spheres_on_cell_edges(prec):
    # spheres exactly on lower cell corners and just below upper corners (in
    # binary32 the upper ones round onto the face and are clamped below it)
    w, n = 1.1, 4
    L = [n * w] * 3
    lo = [[i * w, j * w, k * w] for k in (0, 2) for j in (0, 2) for i in (0, 2)]
    hi = [[(i + 1) * w - 1e-12, (j + 1) * w - 1e-12, (k + 1) * w - 1e-12] for k in (0, 2) for j in (0, 2)
          for i in (0, 2)]
    xyz = np.array(lo + hi)
    s = O.System3(len(xyz), L, 1.0, 0.3, 4, 14, prec, xyz=xyz)
    loc, cnt = s.state()
    wl = s.w if prec == O.FP64 else s.w.astype(np.float32).astype(np.float64)
    occ = np.arange(8)[None, :] < cnt[:, None]
    assert all(loc[:, :, a][occ].max() < wl[a] for a in range(3))
    for _ in range(200):
        s.shift()
        assert s.state()[1].sum() == len(xyz)
    loc, cnt = s.state()
    occ = np.arange(8)[None, :] < cnt[:, None]
    assert all(loc[:, :, a][occ].max() < wl[a] and loc[:, :, a][occ].min() >= 0 for a in range(3))
    s.sweep(50)
    rmin = 1.0 if prec == O.FP64 else 1.0 - 1e-6
    assert s.state()[1].sum() == len(xyz) and O.close_pairs3(s.positions(), s.box(), rmin) == 0


def test_thread_count_and_split_runs_do_not_change_results():
    w = W.spheres_n2048_phi045()
    runs = []
    for threads, split in ((1, False), (4, False), (4, True)):
        O.set_threads(threads)
        s = O.System3(w.N, w.L, 1.0, w.d, 4, 15, O.FP64)
        if split:
            s.sweep(3)
            s.sweep(5)
        else:
            s.sweep(8)
        runs.append((s.state()[0], s.counters()))
    O.set_threads(0)
    for loc, cnt in runs[1:]:
        assert np.array_equal(loc, runs[0][0]) and np.array_equal(cnt, runs[0][1])


def test_errors_3d():
    w = W.spheres_n2048_phi045()
    with pytest.raises(O.OracleError):
        O.System3(w.N, w.L, 1.0, 0.6, 4, 1)        # d >= w/2
    with pytest.raises(O.OracleError):
        O.System3(w.N, w.L, 1.0, 0.1, 0, 1)        # n_M = 0
    xyz = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]])
    with pytest.raises(O.OracleError) as e:
        O.System3(2, [6.0] * 3, 1.0, 0.1, 4, 1, xyz=xyz)
    assert e.value.code == O.EOVERLAP
    with pytest.raises(O.OracleError) as e:
        O.System3(2, [6.0] * 3, 1.0, 0.1, 4, 1, xyz=np.array([[1.0, 1.0, 1.0], [7.0, 1.0, 1.0]]))
    assert e.value.code == O.EINVAL


# ---------------------------------------------------------------------------
# Random draws
# ---------------------------------------------------------------------------
def test_decode_perm8_is_a_bijection():
    seen = set()
    for k in range(math.factorial(8)):
        p = tuple(O.decode_perm8(8, k))
        assert sorted(p) == list(range(8))
        seen.add(p)
    assert len(seen) == math.factorial(8)


def test_cell_shuffles_uniform():
    n = 5
    counts = {}
    for c in range(24000):
        p, _ = O.cell_draws3(3, 9, c, 6, n, 1)
        counts[tuple(p)] = counts.get(tuple(p), 0) + 1
    assert len(counts) == 120
    chi2 = stats.chisquare(list(counts.values()))
    assert chi2.pvalue > 1e-4


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_ball_directions_uniform(prec):
    u = np.vstack([O.cell_draws3(5, 3, c, 2, 1, 8, precision=prec)[1] for c in range(4000)])
    r = np.linalg.norm(u, axis=1)
    assert r.max() < 1.0
    assert stats.kstest(r**3, "uniform").pvalue > 1e-4
    assert stats.kstest((u[:, 2] / r + 1) / 2, "uniform").pvalue > 1e-4
    phi = (np.arctan2(u[:, 1], u[:, 0]) + math.pi) / (2 * math.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-4
    # each trial's draws do not depend on the cell's population
    a = O.cell_draws3(5, 3, 17, 2, 1, 8, precision=prec)[1]
    b = O.cell_draws3(5, 3, 17, 2, 7, 8, precision=prec)[1]
    assert np.array_equal(a, b)
    # mirror symmetry of the variates: the lattices are symmetric about 0
    if prec == O.FP32:
        assert np.all(np.abs(u) * 2**21 % 2 == 1)          # odd multiples of 2^-21
    else:
        assert np.all(np.abs(u) * 2**52 % 2 == 1)          # odd multiples of 2^-52


def test_binary32_directions_are_the_21bit_field_triples():
    # attempts come from block b's fields (0,1,2) and (3,4,5) in order; with
    # rejections the kept ones are a subsequence of the attempts
    seed, sweep, cell, Q = 9, 4, 33, 6
    kept = O.cell_draws3(seed, sweep, cell, Q, 1, 12, precision=O.FP32)[1]
    attempts = []
    for b in range(40):
        f = O.fields21(O.philox([sweep, cell, (1 << 28) | (Q << 24), b], [seed & 0xFFFFFFFF, seed >> 32]))
        for t in range(2):
            a = np.array([(2 * int(x) + 1 - 2**21) * 2.0**-21 for x in f[3 * t:3 * t + 3]])
            attempts.append(a)
    inside = [a for a in attempts if (a**2).sum() < 1 - 1e-6]
    assert np.array_equal(kept, np.array(inside[:12]))


def test_sweep_draws3():
    w = np.array([1.01, 1.02, 1.03])
    first, dirs = [], []
    for s in range(6000):
        perm, f, ds = O.sweep_draws3(21, s, w)
        assert sorted(perm) == list(range(8))
        assert 0 <= f < 6 and 0 <= ds < w[f >> 1] / 2
        first.append(perm[0])
        dirs.append(f)
    assert stats.chisquare(np.bincount(first, minlength=8)).pvalue > 1e-4
    assert stats.chisquare(np.bincount(dirs, minlength=6)).pvalue > 1e-4


# ---------------------------------------------------------------------------
# Stationary distribution
# ---------------------------------------------------------------------------
def test_two_spheres_sample_the_uniform_distribution():
    # the separation of two spheres on a 4^3 torus is uniform over the cube
    # [-2,2)^3 minus the ball |r| < sigma
    L = 4.0
    s = O.System3(2, [L] * 3, 1.0, 0.45, 4, 2025, O.FP64,
                  xyz=np.array([[0.5, 0.5, 0.5], [2.5, 2.5, 2.5]]))
    s.sweep(200)
    seps = []
    for _ in range(30000):
        s.sweep(6)
        p = s.positions()
        seps.append(_min_image(p[1] - p[0], L))
    seps = np.array(seps)
    r = np.linalg.norm(seps, axis=1)
    assert r.min() >= 1.0 - 1e-12
    inside = r < 2.0
    p_in = (4 * math.pi / 3) * 7 / (64 - 4 * math.pi / 3)
    n_eff = len(r) / 4
    assert abs(inside.mean() - p_in) < 4 * math.sqrt(p_in * (1 - p_in) / n_eff)
    ri = r[inside]
    assert stats.kstest((ri**3 - 1) / 7, "uniform").statistic < 1.6 / math.sqrt(len(ri) / 4)
    # unordered pair: the separation's direction is defined up to sign
    cz = np.abs(seps[inside, 2] / ri)
    assert stats.kstest(cz, "uniform").statistic < 1.6 / math.sqrt(len(ri) / 4)
    # the density of the separation is flat away from the ball: in each slab
    # |s_a| >= 1.2 (wholly outside it) the folded components are uniform
    a_s = np.abs(seps)
    for a in range(3):
        slab = a_s[a_s[:, a] >= 1.2]
        crit = 1.6 / math.sqrt(len(slab) / 4)
        assert stats.kstest((slab[:, a] - 1.2) / 0.8, "uniform").statistic < crit
        for b in range(3):
            if b != a:
                assert stats.kstest(slab[:, b] / 2, "uniform").statistic < crit


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_four_spheres_match_rejection_sampling(prec):
    L = 4.4
    rng = np.random.default_rng(9)
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)]

    def min_dist(p):
        return min(np.linalg.norm(_min_image(p[i] - p[j], L)) for i, j in pairs)

    ref = []
    while len(ref) < 20000:
        p = rng.uniform(0, L, (4, 3))
        dm = min_dist(p)
        if dm >= 1.0:
            ref.append(dm)
    start = np.array([[0.5, 0.5, 0.5], [2.7, 0.5, 0.5], [0.5, 2.7, 2.7], [2.7, 2.7, 0.5]])
    s = O.System3(4, [L] * 3, 1.0, 0.4, 4, 78, prec, xyz=start)
    s.sweep(200)
    mc = []
    for _ in range(12000):
        s.sweep(5)
        mc.append(min_dist(s.positions()))
    res = stats.ks_2samp(np.array(ref), np.array(mc))
    n_eff = len(mc) / 3
    assert res.statistic < 1.95 * math.sqrt(1 / n_eff + 1 / len(ref))


# ---------------------------------------------------------------------------
# Contact histogram and pressure in three dimensions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_histogram3_equals_brute_force(prec):
    w = W.spheres_n2048_phi045()
    s = O.System3(w.N, w.L, 1.0, w.d, 4, 16, prec)
    s.sweep(30)
    h = s.histogram(200, 1e-4)
    hb = O.bruteforce_histogram3(s.positions(), s.box(), 1.0, 200, 1e-4)
    assert h.sum() > 100 and h.sum() % 2 == 0
    assert np.array_equal(h, hb)


def _pair_histogram3_kdtree(xyz, L, sigma, nbins, dr):
    from scipy.spatial import cKDTree
    t = cKDTree(xyz, boxsize=L)
    pairs = t.query_pairs(sigma + nbins * dr, output_type="ndarray")
    d = _min_image(xyz[pairs[:, 0]] - xyz[pairs[:, 1]], np.asarray(L))
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    e = sigma + np.arange(nbins + 1) * dr
    E = e * e
    keep = (r2 >= E[0]) & (r2 < E[-1])
    b = np.searchsorted(E, r2[keep], side="right") - 1
    return 2 * np.bincount(b, minlength=nbins)


def test_bruteforce_histogram3_matches_kdtree():
    L = [11.0, 12.0, 13.0]
    xyz = W.uniform_points3(1500, L, 6)
    a = O.bruteforce_histogram3(xyz, L, 1.0, 200, 1e-4)
    b = _pair_histogram3_kdtree(xyz, L, 1.0, 200, 1e-4)
    assert a.sum() > 0 and np.array_equal(a, b)


def test_ideal_gas_contact_value_is_one_3d():
    L = [40.0, 40.0, 40.0]
    N = 40000
    nconf = 8
    hist = np.zeros(200)
    for k in range(nconf):
        hist += _pair_histogram3_kdtree(W.uniform_points3(N, L, 300 + k), L, 1.0, 200, 1e-4)
    R, g = P.g_of_r3(hist, nconf, N, 64000.0, 1.0, 1e-4)
    assert abs(g.mean() - 1) < 4 / math.sqrt(hist.sum() / 2)
    g0 = P.contact_value(R, g, 1.0, 0.02)
    assert abs(g0 - 1) < 4 * 6 / math.sqrt(hist.sum() / 2)


def test_pressure3_closed_form():
    # g = 1 gives beta P / rho = 1 + B2 rho with B2 = 2 pi sigma^3 / 3
    r = P.bin_edges(1.0, 1e-4, 200)
    n = (4 * math.pi / 3) * (r[1:] ** 3 - r[:-1] ** 3)
    bp, g0, pstar = P.pressure3(n, 1, 1, 1.0)
    assert abs(g0 - 1) < 1e-6 and abs(bp - (1 + 2 * math.pi / 3)) < 1e-6
    assert abs(pstar - bp) < 1e-12
    # the sample point is the mean radius of the shell
    R = P.sample_points3(1.0, 0.5, 1)
    x = np.linspace(1.0, 1.5, 200001)
    assert abs(R[0] - np.trapezoid(x**3, x) / np.trapezoid(x**2, x)) < 1e-9


def test_estimator3_on_model_distribution():
    g = keyvals("estimator_sec4.txt")
    amp, rate, dr = g["model_amplitude"], g["model_rate"], g["dr"]
    r = P.bin_edges(1.0, dr, 200)
    # n(r) = 4 pi r^2 g_m(r), g_m = amp exp(-rate (r - 1)), integrated over each bin
    x = np.linspace(0, 1, 2001)
    n = np.array([np.trapezoid(4 * np.pi * (lo + (hi - lo) * x) ** 2 * amp * np.exp(-rate * (lo + (hi - lo) * x - 1)),
                               lo + (hi - lo) * x) for lo, hi in zip(r[:-1], r[1:])])
    R, gr = P.g_of_r3(n, 1, 1, 1.0, 1.0, dr)
    g0 = P.contact_value(R, gr, 1.0, g["c"], g["degree"])
    assert abs(g0 / amp - 1) < g["max_relative_bias"]
    # a second least-squares routine gives the same intercept
    keep = (R > 1.0) & (R <= 1.0 + g["c"])
    alt = np.polyval(np.polyfit((R[keep] - 1.0) / g["c"], gr[keep], g["degree"]), 0.0)
    assert abs(alt - g0) < 1e-9 * amp
    # and the pressure formula uses it: beta P / rho = 1 + (2 pi / 3) rho g0
    bp, g0b, _ = P.pressure3(n, 1, 1, 1.0, 1.0, dr, g["c"])
    assert abs(g0b - g0) < 1e-12 and abs(bp - (1 + 2 * math.pi / 3 * g0)) < 1e-12


@pytest.mark.slow
def test_low_density_virial_series_3d():
    # hard spheres: beta P / rho = 1 + b rho + B3 rho^2 + B4 rho^3 + B5 rho^4,
    # b = 2 pi sigma^3 / 3, B3 = 5 b^2 / 8, B4 = 0.2869495 b^3, B5 = 0.110252 b^4
    w = W.fcc3(8, 0.10, 0.3)
    rho = w.N / np.prod(w.L)
    b = 2 * math.pi / 3
    series = 1 + b * rho + 0.625 * (b * rho) ** 2 + 0.2869495 * (b * rho) ** 3 + 0.110252 * (b * rho) ** 4
    s = O.System3(w.N, w.L, 1.0, w.d, 4, 41, O.FP64)
    s.sweep(200)
    blocks = []
    for _ in range(16):
        h = np.zeros(200)
        for _ in range(500):
            s.sweep(1)
            h += s.histogram(200, 1e-4)
        blocks.append(P.pressure3(h, 500, w.N, float(np.prod(w.L)))[0])
    blocks = np.array(blocks)
    mean, se = blocks.mean(), blocks.std(ddof=1) / math.sqrt(len(blocks))
    assert abs(mean - series) < 3 * se + 2e-3, (mean, se, series)
