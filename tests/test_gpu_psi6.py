"""The library's psi_6 kernel against the oracle: every disk's psi_6 is the
same number (same pairs, same order, every binary64 operation rounded as
written); the means differ only by the order of the sum over disks."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PREC = {"fp64": O.FP64, "fp32": O.FP32}
RCUT = 1.4


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["n1024", "n65536"])
def test_psi6_matches_oracle(prec, case):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070() if case == "n1024" else W.n65536_phi070()
    sweeps = 30 if case == "n1024" else 5
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 9, prec)
    o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 9, PREC[prec])
    g.sweep(sweeps)
    o.sweep(sweeps)
    mean, mabs, mnb, psi = g.psi6(RCUT, per_disk=True)
    ref, ref_psi = o.psi6(RCUT, per_disk=True)
    assert np.array_equal(psi, ref_psi)
    N = w.N
    assert mnb == ref[3] / N
    assert abs(mean.real - ref[0] / N) < 1e-12 and abs(mean.imag - ref[1] / N) < 1e-12
    assert abs(mabs - ref[2] / N) < 1e-12
    # deterministic: the block sums are reduced in a fixed order
    assert g.psi6(RCUT) == (mean, mabs, mnb)


def test_psi6_of_a_lattice_on_the_gpu():
    from paper_1211_1646_gb300 import hdmc
    a, nx, ny = 1.1, 16, 16
    h = a * math.sqrt(3) / 2
    xy = np.array([((i + 0.25 + 0.5 * (j % 2)) * a, (j + 0.5) * h) for j in range(ny) for i in range(nx)])
    s = hdmc.System(nx * ny, nx * a, ny * h, 1.0, 0.1, 4, 1, "fp64", xy=xy)
    mean, mabs, mnb = s.psi6(RCUT)
    assert abs(mean - 1.0) < 1e-12 and abs(mabs - 1.0) < 1e-12 and mnb == 6.0


def test_psi6_rejects_a_cutoff_beyond_two_cells():
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    s = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 1, "fp32")
    wmin = min(float(np.float32(s.wx)), float(np.float32(s.wy)))
    s.psi6(2 * wmin)
    for bad in (0.0, -1.0, 2 * wmin * (1 + 1e-12)):
        with pytest.raises(hdmc.HDMCError) as e:
            s.psi6(bad)
        assert e.value.code == hdmc.HDMC_EINVAL
