"""Pressure estimator of Sec. 4 (Eqs. P, gR, R), written out in numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

From a histogram n[r_i] of ordered pair distances in bins [r_i, r_i + dr),
r_i = sigma + i*dr:
  R_i    = (2/3) (r_{i+1}^3 - r_i^3) / (r_{i+1}^2 - r_i^2)          (Eq. R)
  g(R_i) = n[r_i] / (n_conf * N * rho * 2 pi R_i dr)                  (Eq. gR)
  g(sigma+) = value at r = sigma of the least-squares polynomial of
              degree 5 through (R_i, g(R_i)) over (sigma, sigma + c]
  P* = sigma^2 rho (1 + (pi/2) sigma^2 rho g(sigma+))                 (Eq. P)
The histogram counts ordered pairs; with that count Eq. gR is normalised so
that an ideal gas gives g = 1 (reading of "number of particle pairs").
The polynomial is fitted in the scaled variable t = (R - sigma)/c, which is a
change of basis only (the fitted function is the same).

Three dimensions (hard spheres; the paper states the estimator for disks):
the shell of bin i has volume (4 pi/3)(r_{i+1}^3 - r_i^3), the sample point
is its mean radius R_i = (3/4)(r_{i+1}^4 - r_i^4)/(r_{i+1}^3 - r_i^3), an
ideal gas gives n[r_i] = n_conf N rho (4 pi/3)(r_{i+1}^3 - r_i^3), and the
virial pressure is beta P / rho = 1 + (2 pi/3) rho sigma^3 g(sigma+).
"""
import numpy as np

DR = 1.0e-4     # histogram bin width in units of sigma (Sec. 4)
C_RANGE = 0.02  # fit range c in units of sigma (Sec. 4)
DEGREE = 5      # polynomial degree (Sec. 4)


def bin_edges(sigma: float, dr: float, nbins: int) -> np.ndarray:
    return sigma + dr * np.arange(nbins + 1, dtype=np.float64)


def sample_points(sigma: float, dr: float, nbins: int) -> np.ndarray:
    r = bin_edges(sigma, dr, nbins)
    lo, hi = r[:-1], r[1:]
    return (2.0 / 3.0) * (hi**3 - lo**3) / (hi**2 - lo**2)


def g_of_r(hist, n_conf: int, N: int, area: float, sigma: float, dr: float):
    hist = np.asarray(hist, dtype=np.float64)
    R = sample_points(sigma, dr, hist.size)
    rho = N / area
    g = hist / (n_conf * N * rho * 2.0 * np.pi * R * dr)
    return R, g


def contact_value(R, g, sigma: float, c: float, degree: int = DEGREE) -> float:
    R = np.asarray(R, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    keep = (R > sigma) & (R <= sigma + c)
    t = (R[keep] - sigma) / c
    V = np.vander(t, degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V, g[keep], rcond=None)
    return float(coef[0])


def pressure(hist, n_conf: int, N: int, area: float, sigma: float = 1.0,
             dr: float = DR, c: float = C_RANGE):
    """Returns (betaP_over_rho, g_contact, P_star)."""
    R, g = g_of_r(hist, n_conf, N, area, sigma, dr)
    g0 = contact_value(R, g, sigma, c)
    rho = N / area
    bp = 1.0 + 0.5 * np.pi * rho * sigma * sigma * g0
    return bp, g0, rho * sigma * sigma * bp


def sample_points3(sigma: float, dr: float, nbins: int) -> np.ndarray:
    r = bin_edges(sigma, dr, nbins)
    lo, hi = r[:-1], r[1:]
    return 0.75 * (hi**4 - lo**4) / (hi**3 - lo**3)


def g_of_r3(hist, n_conf: int, N: int, volume: float, sigma: float, dr: float):
    hist = np.asarray(hist, dtype=np.float64)
    r = bin_edges(sigma, dr, hist.size)
    R = sample_points3(sigma, dr, hist.size)
    rho = N / volume
    g = hist / (n_conf * N * rho * (4.0 * np.pi / 3.0) * (r[1:] ** 3 - r[:-1] ** 3))
    return R, g


def pressure3(hist, n_conf: int, N: int, volume: float, sigma: float = 1.0,
              dr: float = DR, c: float = C_RANGE):
    """Hard spheres: returns (betaP_over_rho, g_contact, P* = rho sigma^3 betaP/rho)."""
    R, g = g_of_r3(hist, n_conf, N, volume, sigma, dr)
    g0 = contact_value(R, g, sigma, c)
    rho = N / volume
    bp = 1.0 + (2.0 * np.pi / 3.0) * rho * sigma**3 * g0
    return bp, g0, rho * sigma**3 * bp
