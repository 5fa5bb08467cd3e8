"""The bounds-checked debug build (-DHDMC_CHECK, the substitute for
compute-sanitizer): every cell index the kernels compute is checked against
the grid.  Run here in a separate process on the disk and sphere paths
(single systems of both precisions with ragged grids, a batch, explicit
shifts and histograms), it must report no failed check and give results
bit-identical to the oracle, like the product build.  (A failing check is
not provoked on purpose: that would need a kernel with a planted bad index.)
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import sys
    import numpy as np
    sys.path.insert(0, %r)
    import oracle as O
    from paper_1211_1646_gb300 import build, hdmc, workloads as W

    lib = build.build(check=True)
    hdmc.library_path = lambda: lib
    assert hdmc.hdmc_build_flags() == hdmc.HDMC_BUILD_CHECK
    O.set_threads(4)
    PREC = {"fp64": O.FP64, "fp32": O.FP32}

    # disks: the 1024-disk workload and a ragged 36 x 22 grid, both precisions
    cases = [W.n1024_phi070(), W.Workload("ragged", 600, 38.5, 23.1, 0.12, 7, 5, 0)]
    for w in cases:
        for prec in ("fp64", "fp32"):
            g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, prec)
            o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, PREC[prec])
            g.sweep(30); o.sweep(30)
            g.shift(); o.shift()
            assert np.array_equal(g.state()[0], o.state()[0]), (w.name, prec)
            assert np.array_equal(g.counters(), o.counters())
            g.sample()
            assert np.array_equal(g.pressure()[2], o.histogram())
            g.psi6(1.4)
            g.close()

    # a batch of three replicas of different size, density and n_M
    reps = [W.Workload("a", 1024, *W.square_box(1024, 0.70), 0.15, 4, 11, 0),
            W.Workload("b", 600, 38.5, 23.1, 0.12, 7, 12, 0),
            W.Workload("c", 2048, *W.square_box(2048, 0.66), 0.1, 3, 13, 0)]
    b = hdmc.Batch(reps, precision="fp32")
    b.sweep(20)
    b.sample()
    b.pressure()
    for r, w in enumerate(reps):
        o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, w.seed, O.FP32)
        o.sweep(20)
        assert np.array_equal(b.state(r)[0], o.state()[0]), w.name
    b.close()

    # spheres: 2048 spheres and an uneven 12 x 10 x 10 grid, both precisions
    w3 = W.spheres_n2048_phi045()
    L2 = [13.3, 10.6, 11.9]
    xyz2 = O.lattice3_positions(864, [13.3] * 3, 1.0, 3) * (np.array(L2) / 13.3)
    for prec in ("fp64", "fp32"):
        for N, L, d, xyz in ((w3.N, w3.L, w3.d, None), (864, L2, 0.1, xyz2)):
            g = hdmc.System3(N, L, 1.0, d, 5, 17, prec, xyz=xyz)
            o = O.System3(N, L, 1.0, d, 5, 17, PREC[prec], xyz=xyz)
            g.sweep(12); o.sweep(12)
            g.shift(); o.shift()
            assert np.array_equal(g.state()[0], o.state()[0]), (N, prec)
            assert np.array_equal(g.counters(), o.counters())
            g.sample()
            assert np.array_equal(g.pressure()[2], o.histogram())
            g.close()
    print("checked build ok")
''') % ROOT


def test_checked_build_reports_no_bad_index_and_matches_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
