"""Pins of the oracle's bond-orientational order psi_6 (the order parameter
whose autocorrelation time Sec. 3.3 minimises): exact values on lattices,
the symmetry of a mirror image, and brute force over all pairs and periodic
images of global coordinates."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def built():
    from oracle import build
    build.build()


A = 1.1          # lattice spacing (sigma = 1)
RCUT = 1.4       # between the first (A) and second (sqrt(3) A, sqrt(2) A) shells


def triangular(nx, ny, rows_along_x=True):
    """nx x ny triangular lattice (ny even) filling its periodic box."""
    h = A * math.sqrt(3) / 2
    xy = np.array([((i + 0.25 + 0.5 * (j % 2)) * A, (j + 0.5) * h) for j in range(ny) for i in range(nx)])
    L = (nx * A, ny * h)
    if not rows_along_x:
        xy = xy[:, ::-1].copy()
        L = L[::-1]
    return xy, L


def square(n):
    xy = np.array([((i + 0.25) * A, (j + 0.25) * A) for j in range(n) for i in range(n)])
    return xy, (n * A, n * A)


def _system(xy, L, prec=O.FP64):
    return O.System(len(xy), L[0], L[1], 1.0, 0.1, 4, 1, prec, xy=xy)


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_triangular_lattice_is_perfectly_ordered(prec):
    xy, L = triangular(16, 16)
    s = _system(xy, L, prec)
    out = s.psi6(RCUT)
    N = len(xy)
    assert out[3] == 6 * N                       # six neighbours each
    assert abs(out[0] / N - 1.0) < 1e-12 and abs(out[1] / N) < 1e-12
    assert abs(out[2] / N - 1.0) < 1e-12


def test_lattice_turned_by_90_degrees_gives_minus_one():
    # bonds at 30 + 60 k degrees: exp(6 i theta) = exp(i pi) = -1
    xy, L = triangular(16, 16, rows_along_x=False)
    s = _system(xy, L)
    out = s.psi6(RCUT)
    N = len(xy)
    assert out[3] == 6 * N
    assert abs(out[0] / N + 1.0) < 1e-12 and abs(out[1] / N) < 1e-12


def test_square_lattice_has_no_sixfold_order():
    # four bonds at 0, 90, 180, 270 degrees: 1 - 1 + 1 - 1 = 0
    xy, L = square(16)
    s = _system(xy, L)
    out, psi = s.psi6(RCUT, per_disk=True)
    N = len(xy)
    assert out[3] == 4 * N
    assert np.abs(psi).max() < 1e-12
    assert abs(out[2]) < 1e-9


def test_mirror_image_conjugates_psi6():
    w_N, L = 1024, (33.8958, 33.8958)
    s = O.System(w_N, L[0], L[1], 1.0, 0.15, 4, 3, O.FP64)
    s.sweep(40)
    xy = s.positions()
    box = s.box()
    mirrored = xy.copy()
    mirrored[:, 0] = np.mod(-mirrored[:, 0], box[0])
    a = O.bruteforce_psi6(xy, box[0], box[1], RCUT)[0]
    b = O.bruteforce_psi6(mirrored, box[0], box[1], RCUT)[0]
    assert abs(a[1]) > 1.0                       # a configuration with a phase to flip
    assert abs(a[0] - b[0]) < 1e-9 and abs(a[1] + b[1]) < 1e-9 and abs(a[2] - b[2]) < 1e-9
    assert a[3] == b[3]


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_cell_list_equals_brute_force(prec):
    N, L = 1024, (33.8958, 33.8958)
    s = O.System(N, L[0], L[1], 1.0, 0.15, 4, 5, prec)
    s.sweep(60)
    out, psi = s.psi6(RCUT, per_disk=True)
    xy = s.positions()                           # canonical (cell, slot) order
    ref, ref_psi = O.bruteforce_psi6(xy, *s.box(), RCUT)
    loc, cnt = s.state()
    occ = np.arange(4)[None, :] < cnt[:, None]
    assert out[3] == ref[3]
    np.testing.assert_allclose(psi[occ], ref_psi, rtol=0, atol=1e-9)
    np.testing.assert_allclose(out[:3], ref[:3], rtol=0, atol=1e-7)


def test_single_bond_at_15_degrees_gives_plus_i():
    # each of the two disks sees its only neighbour at 15 or 195 degrees:
    # exp(6 i theta) = exp(i pi / 2) = i for both (pins the sign of the
    # imaginary part and the power 6)
    t = math.radians(15.0)
    xy = np.array([[4.0, 4.0], [4.0 + 1.2 * math.cos(t), 4.0 + 1.2 * math.sin(t)]])
    s = _system(xy, (10.0, 10.0))
    out, psi = s.psi6(RCUT, per_disk=True)
    assert out[3] == 2
    assert abs(out[0]) < 1e-12 and abs(out[1] - 2.0) < 1e-12
    ref, ref_psi = O.bruteforce_psi6(xy, 10.0, 10.0, RCUT)
    np.testing.assert_allclose(ref_psi, [[0.0, 1.0], [0.0, 1.0]], atol=1e-12)
