"""Balance controls of Table 1 (Sec. 2.4) and move-size tuning (Sec. 3.3)
through the C ABI.

With a control switched off, the library must still be the oracle with the
same switch, bit for bit (the controls change what the chain does with its
random numbers, not which numbers it draws).  The move-size tuner is host
logic over sweeps and counters: replaying its rule on the oracle must give
the same d and the same state.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PREC = {"fp64": O.FP64, "fp32": O.FP32}
COMBOS = [(False, True), (True, False), (False, False)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


def _same(g, o):
    lg, cg = g.state()
    lo, co = o.state()
    assert np.array_equal(cg, co)
    assert np.array_equal(lg, lo)
    assert np.array_equal(g.counters(), o.counters())
    assert np.array_equal(g.origin(), o.origin())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("particles,sets", COMBOS)
def test_controls_match_oracle(prec, particles, sets):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 21, prec)
    o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 21, PREC[prec])
    g.sweep(7)
    o.sweep(7)
    g.set_balance(particles, sets)
    o.set_balance(particles, sets)
    g.sweep(60)
    o.sweep(60)
    _same(g, o)
    # and back on: the method again
    g.set_balance(True, True)
    o.set_balance(True, True)
    g.sweep(9)
    o.sweep(9)
    _same(g, o)


def test_controls_change_the_trajectory():
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    runs = {}
    for combo in [(True, True)] + COMBOS:
        s = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 5, "fp32")
        s.set_balance(*combo)
        s.sweep(20)
        runs[combo] = s.state()[0]
    keys = list(runs)
    for a in range(len(keys)):
        for b in range(a + 1, len(keys)):
            assert not np.array_equal(runs[keys[a]], runs[keys[b]]), (keys[a], keys[b])


def test_batch_controls_per_replica():
    from paper_1211_1646_gb300 import hdmc
    Lx, Ly = W.square_box(1024, 0.70)
    reps = [W.Workload("r%d" % k, 1024, Lx, Ly, 0.15, 4, 40 + k, 0) for k in range(4)]
    flags = [(True, True)] + COMBOS
    b = hdmc.Batch(reps, precision="fp32")
    b.set_balance([f[0] for f in flags], [f[1] for f in flags])
    b.sweep(40)
    for r, (w, f) in enumerate(zip(reps, flags)):
        o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, w.seed, O.FP32)
        o.set_balance(*f)
        o.sweep(40)
        assert np.array_equal(b.state(r)[0], o.state()[0]), f
        assert np.array_equal(b.counters()[r], o.counters()), f


def _oracle_tune(o, d, target, sweeps, every, wx, wy, sigma=1.0):
    """The tuning rule of hdmc_tune_move_size, replayed on the oracle."""
    dmax, dmin = 0.49 * min(wx, wy), 1e-6 * sigma
    c0 = o.counters()
    done = 0
    while done < sweeps:
        o.sweep(min(every, sweeps - done))
        c1 = o.counters()
        tr, ac = int(c1[0]) - int(c0[0]), int(c1[1]) - int(c0[1])
        f = 2.0 if tr == 0 else math.sqrt((ac / tr) / target)
        f = min(max(f, 0.5), 2.0)
        d = min(max(d * f, dmin), dmax)
        o.set_move_size(d)
        c0 = c1
        done += every
    return d


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tune_move_size_matches_oracle_and_hits_target(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, 0.05, 4, 8, prec)
    o = O.System(w.N, w.Lx, w.Ly, 1.0, 0.05, 4, 8, PREC[prec])
    d_gpu = g.tune_move_size(0.30, 1000, 100)
    d_orc = _oracle_tune(o, 0.05, 0.30, 1000, 100, g.wx, g.wy)
    assert d_gpu == d_orc
    _same(g, o)
    c0 = g.counters()
    g.sweep(400)
    c1 = g.counters()
    acc = (int(c1[1]) - int(c0[1])) / (int(c1[0]) - int(c0[0]))
    assert abs(acc - 0.30) < 0.03, acc


def test_tune_move_size_rejects_bad_arguments():
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 8, "fp32")
    for args in [(0.0, 100, 10), (1.0, 100, 10), (0.3, 0, 10), (0.3, 100, 0)]:
        with pytest.raises(hdmc.HDMCError) as e:
            g.tune_move_size(*args)
        assert e.value.code == hdmc.HDMC_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_snapshot_carries_controls(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    a = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 31, prec)
    a.set_balance(False, False)
    a.sweep(10)
    img = a.save()
    b = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 31, prec)
    b.load(img)
    a.sweep(25)
    b.sweep(25)
    assert np.array_equal(a.state()[0], b.state()[0])
    o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 31, PREC[prec])
    o.set_balance(False, False)
    o.sweep(35)
    assert np.array_equal(b.state()[0], o.state()[0])
