"""Batched replicas through the C ABI.

A replica of a batch is, by construction, the system hdmc_create builds from
the same arguments: its trajectory must be bit-identical to the single-system
run (and so to the oracle), whatever the block layout of the batched launches.
"""
import numpy as np
import pytest

import oracle as O
from oracle import pressure as P
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _replicas():
    Lx1, Ly1 = W.square_box(1024, 0.70)
    nx, ny = W.hex_counts(2048)
    Lx3, Ly3 = W.hex_box(nx, ny, 0.65)
    Lx4, Ly4 = W.hex_box(64, 64, 0.72)
    return [
        W.Workload("a", 1024, Lx1, Ly1, 0.15, 4, 11, 0),
        W.Workload("b", 600, 37.3, 23.9, 0.2, 7, 12, 0),        # ragged 36 x 22 grid
        W.Workload("c", nx * ny, Lx3, Ly3, 0.1, 2, 13, 0),
        W.Workload("d", 4096, Lx4, Ly4, 0.08, 1, 14, 0),
    ]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


def _singles(reps, prec):
    from paper_1211_1646_gb300 import hdmc
    return [hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, prec) for w in reps]


def _same_as_singles(b, singles):
    cnt_b = b.counters()
    for r, s in enumerate(singles):
        lb, cb = b.state(r)
        ls, cs = s.state()
        assert np.array_equal(cb, cs), "replica %d counts" % r
        assert np.array_equal(lb, ls), "replica %d positions" % r
        assert np.array_equal(cnt_b[r], s.counters()), "replica %d counters" % r
        assert np.array_equal(b.origin(r), s.origin()), "replica %d origin" % r


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_equals_single_systems(prec):
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision=prec)
    singles = _singles(reps, prec)
    b.sweep(70)                      # one 64-sweep graph plus a 6-sweep graph
    for s in singles:
        s.sweep(70)
    _same_as_singles(b, singles)


def test_batch_block_layout_does_not_change_results():
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision="fp32")
    singles = _singles(reps, "fp32")
    for rows in (2, 8, 1, 4, 2):
        b.set_rows(rows)
        b.sweep(9)
        for s in singles:
            s.sweep(9)
        _same_as_singles(b, singles)
    assert b.config()[0] == 2


def test_batch_matches_oracle_and_pressure():
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision="fp32")
    orcs = [O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, O.FP32) for w in reps]
    b.sweep(12)
    b.sample()
    for o in orcs:
        o.sweep(12)
    bp, g0, hist, ns = b.pressure()
    assert ns == 1
    for r, (w, o) in enumerate(zip(reps, orcs)):
        assert np.array_equal(b.state(r)[0], o.state()[0])
        h = o.histogram()
        assert np.array_equal(hist[r], h)
        bp_ref, _, _ = P.pressure(h, 1, w.N, w.Lx * w.Ly)
        assert abs(bp[r] - bp_ref) < 1e-9 * abs(bp_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_paper_cell_rule(prec):
    # replicas with the Sec. 3.1 cells (just below sqrt(2) sigma), each the
    # oracle's chain on that grid, bit for bit
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision=prec, cells="sqrt2")
    orcs = [O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, O.FP64 if prec == "fp64" else O.FP32,
                     cells=O.CELLS_SQRT2) for w in reps]
    for r, o in enumerate(orcs):
        assert (b.grids[r]["mx"], b.grids[r]["my"]) == (o.mx, o.my)
    b.sweep(20)
    for o in orcs:
        o.sweep(20)
    for r, o in enumerate(orcs):
        assert np.array_equal(b.state(r)[1], o.state()[1])
        assert np.array_equal(b.state(r)[0], o.state()[0])
        assert np.array_equal(b.counters()[r], o.counters())


@pytest.mark.parametrize("rows,common", [(1, None), (8, None), (2, 4), (4, 8)])
def test_batch_crowded_cells(rows, common):
    # every replica with cells of 1.3 disks or more on average (Sec. 3.1
    # cells, phi >= 0.62): the batch runs the binary32 crowded-cell
    # sub-sweep, with four different n_M or one n_M shared by every replica
    # (4 or 8: a kernel with n_M fixed), bit for bit with the oracle
    from paper_1211_1646_gb300 import hdmc
    reps = []
    for i, (nx, ny, phi, nsel) in enumerate([(40, 36, 0.62, 1), (33, 50, 0.68, 2), (64, 64, 0.72, 8),
                                             (27, 22, 0.74, 3)]):
        Lx, Ly = W.hex_box(nx, ny, phi)
        reps.append(W.Workload("crowded%d" % i, nx * ny, Lx, Ly, 0.12, common or nsel, 41 + i, 0))
    b = hdmc.Batch(reps, precision="fp32", cells="sqrt2")
    b.set_rows(rows)
    orcs = [O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, O.FP32, cells=O.CELLS_SQRT2) for w in reps]
    for r, (w, o) in enumerate(zip(reps, orcs)):
        assert (b.grids[r]["mx"], b.grids[r]["my"]) == (o.mx, o.my)
        assert 10 * w.N >= 13 * o.mx * o.my   # the library's crowded-cell rule
    b.sweep(12)
    for o in orcs:
        o.sweep(12)
    for r, o in enumerate(orcs):
        assert np.array_equal(b.state(r)[1], o.state()[1])
        assert np.array_equal(b.state(r)[0], o.state()[0])
        assert np.array_equal(b.counters()[r], o.counters())


@pytest.mark.parametrize("common", [4, 8])
def test_batch_common_nselect(common):
    # One n_M shared by every replica selects a binary32 kernel with n_M
    # fixed.  The batch changes n_M between runs (shared, differing, shared
    # again); each replica must follow a chain of single systems running the
    # same phases (one per phase, started from the state the previous one
    # ended in).
    from paper_1211_1646_gb300 import hdmc
    reps = [W.Workload(w.name, w.N, w.Lx, w.Ly, w.d, common, w.seed, 0) for w in _replicas()]
    b = hdmc.Batch(reps, precision="fp32")
    states = [None] * len(reps)
    for ns in ([common] * 4, [common, 3, common, 1], [common] * 4):
        b.set_nselect(ns)
        b.sweep(9)
        for r, (w, m) in enumerate(zip(reps, ns)):
            s = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, m, w.seed, "fp32")
            if states[r] is not None:
                s.set_state(*states[r])
            s.sweep(9)
            loc, cnt = s.state()
            info = s.info()
            states[r] = (loc, cnt, info["origin"], info["sweeps_done"], info["shifts_done"])
            lb, cb = b.state(r)
            assert np.array_equal(cb, cnt), "n_M %s, replica %d counts" % (ns, r)
            assert np.array_equal(lb, loc), "n_M %s, replica %d positions" % (ns, r)
            assert np.array_equal(b.origin(r), info["origin"]), "n_M %s, replica %d origin" % (ns, r)


def test_batch_autotune_and_invariants():
    from scipy.spatial import cKDTree
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision="fp32")
    rows, nm = b.autotune(16)
    assert rows in (1, 2, 4, 8) and nm in (1, 2, 4, 8)
    assert b.config()[0] == rows and list(b.config()[1]) == [nm] * len(reps)
    b.sweep(40)
    cnt = b.counters()
    for r, w in enumerate(reps):
        loc, c = b.state(r)
        assert int(c.sum()) == w.N and c.max() <= 4
        assert cnt[r, 0] == cnt[r, 1] + cnt[r, 2] + cnt[r, 3]
        g = b.grids[r]
        wx, wy = float(np.float32(g["wx"])), float(np.float32(g["wy"]))
        occ = np.arange(4)[None, :] < c[:, None]
        cx = np.repeat(np.arange(g["mx"] * g["my"]) % g["mx"], 4).reshape(-1, 4)
        cy = np.repeat(np.arange(g["mx"] * g["my"]) // g["mx"], 4).reshape(-1, 4)
        X = (cx * wx + loc[..., 0])[occ]
        Y = (cy * wy + loc[..., 1])[occ]
        org = b.origin(r)
        box = np.array([g["mx"] * wx, g["my"] * wy])
        xy = np.mod(np.stack([X + org[0], Y + org[1]], 1), box)
        assert len(cKDTree(xy, boxsize=box).query_pairs(1.0 - 1e-6)) == 0


def test_batch_of_64_replicas_runs():
    from paper_1211_1646_gb300 import hdmc
    reps = W.batch64()
    b = hdmc.Batch(reps, precision="fp32")
    b.sweep(5)
    b.sample()
    bp, g0, hist, ns = b.pressure()
    assert np.all(np.isfinite(bp)) and np.all(bp > 1.0)
    cnt = b.counters()
    assert np.all(cnt[:, 0] > 0)


def _same_batches(a, b, R):
    ca, cb = a.counters(), b.counters()
    for r in range(R):
        assert np.array_equal(a.state(r)[0], b.state(r)[0]), r
        assert np.array_equal(a.state(r)[1], b.state(r)[1]), r
        assert np.array_equal(ca[r], cb[r]), r
        assert np.array_equal(a.origin(r), b.origin(r)), r


def test_batch_snapshot_resume_is_bit_identical():
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    a = hdmc.Batch(reps, precision="fp32")
    a.sweep(30)
    a.set_rows(2)
    a.set_nselect([3, 5, 2, 4])
    a.set_balance([True, False, True, True], [True, True, False, True])
    a.sweep(10)
    a.sample()
    img = a.save()
    assert img.nbytes == a.snapshot_bytes()
    # a batch of the same replicas with other seeds, d and n_M takes them from the image
    other = [W.Workload(w.name, w.N, w.Lx, w.Ly, 0.05, 1, w.seed + 1000, 0) for w in reps]
    b = hdmc.Batch(other, precision="fp32")
    b.sweep(3)
    b.load(img)
    assert b.config()[0] == 2 and list(b.config()[1]) == [3, 5, 2, 4]
    _same_batches(a, b, len(reps))
    for x in (a, b):
        x.sweep(70)
        x.sample()
    _same_batches(a, b, len(reps))
    pa, pb = a.pressure(), b.pressure()
    assert pa[3] == pb[3] == 2
    assert np.array_equal(pa[2], pb[2]) and np.array_equal(pa[0], pb[0])


def test_batch_snapshot_rejects_bad_images_and_keeps_state():
    import struct
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    src = hdmc.Batch(reps, precision="fp32")
    src.sweep(12)
    good = src.save()
    dst = hdmc.Batch(reps, precision="fp32")
    ref = hdmc.Batch(reps, precision="fp32")
    dst.sweep(5)
    ref.sweep(5)
    off_cells = struct.unpack_from("<Q", bytes(good[72:80]))[0]   # header field off_cells
    bad = good.copy()
    cells = bad[off_cells:].view(np.float32)
    first = int(np.argmax(cells >= 0))          # an occupied x coordinate
    cells[first] = 1e6                          # far outside its cell
    with pytest.raises(hdmc.HDMCError) as e:
        dst.load(bad)
    assert e.value.code == hdmc.HDMC_EINVAL
    short = good[:-1]
    with pytest.raises(hdmc.HDMCError):
        dst.load(short)
    three = hdmc.Batch(reps[:3], precision="fp32")
    with pytest.raises(hdmc.HDMCError):
        three.load(np.resize(good, three.snapshot_bytes()))
    _same_batches(dst, ref, len(reps))
    dst.sweep(7)
    ref.sweep(7)
    _same_batches(dst, ref, len(reps))
    dst.load(good)
    _same_batches(dst, src, len(reps))


def test_batch_psi6_equals_single_systems():
    from paper_1211_1646_gb300 import hdmc
    reps = _replicas()
    b = hdmc.Batch(reps, precision="fp32")
    singles = _singles(reps, "fp32")
    b.sweep(25)
    for s in singles:
        s.sweep(25)
    mean, mabs, mnb = b.psi6(1.4)
    for r, s in enumerate(singles):
        assert (mean[r], mabs[r], mnb[r]) == s.psi6(1.4)
