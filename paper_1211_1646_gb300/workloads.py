"""Seeded synthetic workloads for the hard-disk sweep.

This module only defines inputs: box sizes for a target packing fraction,
the named workload parameters, replica draws for the batched workload and
uniform random points.  It contains none of the Monte Carlo arithmetic, and
both the CUDA library's tests and the CPU oracle take their inputs from it.

Packing fraction phi = N pi sigma^2 / (4 Lx Ly) (Sec. 4).  A hexagonal
lattice of spacing a has area sqrt(3)/2 a^2 per disk, so a = sigma
sqrt(pi / (2 sqrt(3) phi)); an nx x ny hexagonal patch (ny even) tiles the
periodic box nx a by ny a sqrt(3)/2.
"""
import math
from dataclasses import dataclass, field

import numpy as np


def square_box(N: int, phi: float, sigma: float = 1.0):
    L = math.sqrt(N * math.pi * sigma * sigma / (4.0 * phi))
    return L, L


def hex_spacing(phi: float, sigma: float = 1.0) -> float:
    return sigma * math.sqrt(math.pi / (2.0 * math.sqrt(3.0) * phi))


def hex_box(nx: int, ny: int, phi: float, sigma: float = 1.0):
    a = hex_spacing(phi, sigma)
    return nx * a, ny * a * math.sqrt(3.0) / 2.0


def hex_counts(N: int):
    """Near-square hexagonal patch with about N disks: ny even, nx*ny = N'."""
    ny = 2 * max(1, int(round(math.sqrt(N * 2.0 / math.sqrt(3.0)) / 2.0)))
    nx = max(1, int(round(N / ny)))
    return nx, ny


@dataclass
class Workload:
    name: str
    N: int
    Lx: float
    Ly: float
    d: float
    nselect: int
    seed: int
    sweeps: int
    precision: str = "fp64"
    sigma: float = 1.0
    phi: float = 0.0
    extra: dict = field(default_factory=dict)


def n1024_phi070() -> Workload:
    """N=1024 disks, square box, phi=0.70, d=0.15, n_M=4, seed 1, 200 sweeps."""
    Lx, Ly = square_box(1024, 0.70)
    return Workload("n1024_phi0.70_square", 1024, Lx, Ly, 0.15, 4, 1, 200, "fp64", phi=0.70)


def n65536_phi070() -> Workload:
    """N=256^2 disks, square box, phi=0.70, d tuned to ~30% acceptance."""
    Lx, Ly = square_box(65536, 0.70)
    return Workload("n65536_phi0.70_square", 65536, Lx, Ly, 0.10, 4, 1, 10000, "fp64", phi=0.70,
                    extra={"target_acceptance": 0.30, "pressure_every": 100})


def n1m_phi0716(precision: str = "fp32") -> Workload:
    """N=1024^2 disks, hexagonal-aspect box, phi=0.716, d=0.08, n_M=4."""
    Lx, Ly = hex_box(1024, 1024, 0.716)
    return Workload("n1048576_phi0.716_hex", 1024 * 1024, Lx, Ly, 0.08, 4, 1, 100000, precision,
                    phi=0.716)


def n4m(phi: float, precision: str = "fp32") -> Workload:
    """N=2048^2 disks, hexagonal-aspect box, phi in {0.700, 0.710, 0.716, 0.720}."""
    Lx, Ly = hex_box(2048, 2048, phi)
    return Workload("n4194304_phi%.3f_hex" % phi, 2048 * 2048, Lx, Ly, 0.08, 4, 1, 20000, precision, phi=phi)


def paper_table4(precision: str = "fp32") -> Workload:
    """The paper's own throughput workload (Sec. 5.1, Table 4): N = 1520^2
    disks at phi = 0.698 in a square box, cells just below sqrt(2) sigma
    (the paper's cell rule), d = 0.16 and n_M = 4 (the values Sec. 5 finds
    best for the autocorrelation time per second)."""
    Lx, Ly = square_box(1520 * 1520, 0.698)
    return Workload("n2310400_phi0.698_square_sqrt2cells", 1520 * 1520, Lx, Ly, 0.16, 4, 1, 200, precision,
                    phi=0.698, extra={"cells": "sqrt2"})


def batch64(seed: int = 1, R: int = 64, nmin: int = 4096, nmax: int = 262144,
            phimin: float = 0.60, phimax: float = 0.74):
    """Replica list: N log-uniform in [nmin, nmax] (rounded to a hexagonal
    patch), phi uniform in [phimin, phimax], independent 64-bit seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(R):
        Nt = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
        phi = float(rng.uniform(phimin, phimax))
        nx, ny = hex_counts(int(round(Nt)))
        Lx, Ly = hex_box(nx, ny, phi)
        s = int(rng.integers(1, 2**63 - 1))
        out.append(Workload("replica%d" % r, nx * ny, Lx, Ly, 0.08, 4, s, 10000, "fp32", phi=phi))
    return out


def uniform_points(N: int, Lx: float, Ly: float, seed: int) -> np.ndarray:
    """N independent uniform points in [0,Lx) x [0,Ly) (an ideal gas)."""
    rng = np.random.default_rng(seed)
    xy = np.empty((N, 2), dtype=np.float64)
    xy[:, 0] = rng.uniform(0.0, Lx, N)
    xy[:, 1] = rng.uniform(0.0, Ly, N)
    return xy


# ---------------------------------------------------------------------------
# Three dimensions (hard spheres).  Packing fraction phi = N pi sigma^3 /
# (6 V); the start is a face-centred cubic lattice of q^3 unit cells,
# N = 4 q^3, filling a cubic box.
# ---------------------------------------------------------------------------
@dataclass
class Workload3:
    name: str
    N: int
    L: tuple
    d: float
    nselect: int
    seed: int
    sweeps: int
    precision: str = "fp64"
    sigma: float = 1.0
    phi: float = 0.0


def cube_box3(N: int, phi: float, sigma: float = 1.0):
    a = (N * math.pi * sigma**3 / (6.0 * phi)) ** (1.0 / 3.0)
    return (a, a, a)


def fcc3(q: int, phi: float, d: float, seed: int = 1, precision: str = "fp64", nselect: int = 4,
         sweeps: int = 100) -> Workload3:
    N = 4 * q**3
    return Workload3("spheres_n%d_phi%.3f_fcc" % (N, phi), N, cube_box3(N, phi), d, nselect, seed, sweeps,
                     precision, phi=phi)


def spheres_n2048_phi045() -> Workload3:
    """N = 4*8^3 spheres, phi = 0.45 (dense fluid), d = 0.1: 12^3 cells."""
    return fcc3(8, 0.45, 0.10)


def spheres_n16384_phi045() -> Workload3:
    """N = 4*16^3 spheres, phi = 0.45, d = 0.1: 26^3 cells."""
    return fcc3(16, 0.45, 0.10)


def spheres_n1m_phi049(precision: str = "fp32") -> Workload3:
    """N = 4*64^3 = 1,048,576 spheres at the freezing packing fraction
    phi = 0.49, d = 0.08, n_M = 4: 102^3 cells."""
    return fcc3(64, 0.49, 0.08, precision=precision, sweeps=10000)


def uniform_points3(N: int, L, seed: int) -> np.ndarray:
    """N independent uniform points in the box [0,Lx) x [0,Ly) x [0,Lz)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.0, L[a], N) for a in range(3)], axis=1)
