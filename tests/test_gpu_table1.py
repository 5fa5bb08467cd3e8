"""Equation of state against the paper: P* of N = 256^2 hard disks at
phi = 0.716 with the method's shuffles on (Table 1, first row; fixture
tests/golden/balance_table1.txt).

16 independent replicas (binary32, one batch) start from the hexagonal
lattice, equilibrate 5e5 sweeps and sample a contact histogram every 100
sweeps for 1e6 sweeps.  The replicas are independent, so the standard error
of their mean comes from their scatter; the mean must lie within 4 standard
errors (plus the table's own error) of the published value, and the
standard error must be small enough for that to mean something.
"""
import math
import os

import numpy as np
import pytest

from paper_1211_1646_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "balance_table1.txt")
R, NX = 16, 256
EQUIL, SWEEPS, EVERY, BLOCK = 500_000, 1_000_000, 100, 1000


def _table1(phi):
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        p, cb, ph, pstar, two_sigma = line.split()
        if p == "1" and cb == "1" and abs(float(ph) - phi) < 1e-9:
            return float(pstar), float(two_sigma) / 2
    raise KeyError(phi)


def test_pressure_matches_table1_at_phi_0716():
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    phi = 0.716
    ref, ref_se = _table1(phi)
    Lx, Ly = W.hex_box(NX, NX, phi)
    N = NX * NX
    reps = [W.Workload("r%d" % k, N, Lx, Ly, 0.1, 4, 7000 + k, 0) for k in range(R)]
    b = hdmc.Batch(reps, precision="fp32")
    b.sweep(EQUIL)
    acc = np.zeros(R)
    nblocks = 0
    for _ in range(SWEEPS // (EVERY * BLOCK)):
        for _ in range(BLOCK):
            b.sweep(EVERY)
            b.sample()
        bp, _, _, _ = b.pressure()
        acc += bp * N / (Lx * Ly)
        nblocks += 1
    torch.cuda.synchronize()
    per_rep = acc / nblocks
    mean = per_rep.mean()
    se = per_rep.std(ddof=1) / math.sqrt(R)
    print("P*(phi=%.3f) = %.5f +- %.5f (16 replicas); Table 1: %.5f +- %.5f"
          % (phi, mean, se, ref, ref_se))
    assert se < 0.005
    assert abs(mean - ref) <= 4 * se + 2 * ref_se
