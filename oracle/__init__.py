"""Oracle for the checkerboard hard-disk Monte Carlo sweep.

TEST INFRASTRUCTURE ONLY.  This package is the plain, serial, CPU reference
that the CUDA library is checked against.  Only `tests/`, the smoke check in
`__graft_entry__.py` and the CPU-baseline leg of `bench.py` may import it;
the library itself never does, and it never imports the library.

The arithmetic lives in `hdmc_oracle.c` (plain C, binary64 or binary32 as the
mode says, no fused multiply-add except where written as fma()); the
pressure fit of Sec. 4 lives in `pressure.py` (numpy).
"""
import ctypes
import os

import numpy as np

from . import build as _build
from . import pressure  # noqa: F401

OK, EINVAL, EOVERFLOW, EOVERLAP, ENOMEM = 0, 1, 3, 4, 6
FP64, FP32 = 0, 1
EMPTY_SLOT = -1.0e4

_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        sig = {
            "orc_philox": (None, [_u32p, _u32p, _u32p]),
            "orc_stream_bounded": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, _u32p]),
            "orc_stream_words": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int64, _u32p]),
            "orc_lemire_exhaustive": (None, [ctypes.c_uint32, _u64p]),
            "orc_sym52": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_uint32]),
            "orc_grid": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _i32p, _i32p,
                                        _f64p, _f64p]),
            "orc_grid_rule": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _i32p,
                                             _i32p, _f64p, _f64p]),
            "orc_lattice_shape": (ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, _i64p, _i64p]),
            "orc_lattice_positions": (ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_uint64, _f64p]),
            "orc_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_int]),
            "orc_create_from": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_int, _f64p]),
            "orc_destroy": (None, [vp]),
            "orc_set_move_size": (ctypes.c_int, [vp, ctypes.c_double]),
            "orc_set_balance": (None, [vp, ctypes.c_int, ctypes.c_int]),
            "orc_set_allow_leave": (ctypes.c_int, [vp, ctypes.c_int]),
            "orc_set_strips": (ctypes.c_int, [vp, ctypes.c_int]),
            "orc_sweep_phase": (ctypes.c_int, [vp, ctypes.c_int]),
            "orc_strip_start": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "orc_get_row": (None, [vp, ctypes.c_int, _f64p, _u8p]),
            "orc_set_row": (None, [vp, ctypes.c_int, _f64p, _u8p]),
            "orc_sweep_draws": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                       _i32p, _i32p, _f64p]),
            "orc_sweep": (ctypes.c_int, [vp, ctypes.c_int64]),
            "orc_shift": (ctypes.c_int, [vp]),
            "orc_subsweep": (None, [vp, ctypes.c_uint32, ctypes.c_int]),
            "orc_info": (None, [vp, _i32p, _i32p, _f64p, _f64p, _u64p, _u64p]),
            "orc_counters": (None, [vp, _u64p]),
            "orc_origin": (None, [vp, _f64p]),
            "orc_state": (None, [vp, _f64p, _u8p]),
            "orc_positions": (None, [vp, _f64p]),
            "orc_histogram": (None, [vp, ctypes.c_int, ctypes.c_double, _u64p]),
            "orc_psi6": (None, [vp, ctypes.c_double, _f64p, _f64p]),
            "orc_bruteforce_psi6": (None, [_f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _f64p, _f64p]),
            "orc_bruteforce_close_pairs": (ctypes.c_int64, [_f64p, ctypes.c_int64, ctypes.c_double,
                                                            ctypes.c_double, ctypes.c_double]),
            "orc_bruteforce_histogram": (None, [_f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_double, _u64p]),
            "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
            "orc_displacements": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int64, _f64p]),
            "orc_shuffles": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int64, _i32p]),
            "orc_lemire21_exhaustive": (None, [ctypes.c_uint32, _u64p]),
            "orc_sym21": (ctypes.c_float, [ctypes.c_uint32]),
            "orc_fields21": (None, [_u32p, _u32p]),
            "orc_decode_perm": (None, [ctypes.c_int, ctypes.c_uint32, _i32p]),
            "orc_visit_sequence": (None, [ctypes.c_int, ctypes.c_int, _i32p]),
            "orc_local_overlaps": (ctypes.c_int, [vp]),
            "orc_edges2": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_int, _f64p]),
            # three dimensions
            "orc3_decode_perm": (None, [ctypes.c_int, ctypes.c_uint32, _i32p]),
            "orc3_grid": (ctypes.c_int, [_f64p, ctypes.c_double, _i32p, _f64p]),
            "orc3_lattice_positions": (ctypes.c_int, [ctypes.c_int64, _f64p, ctypes.c_double, ctypes.c_uint64,
                                                      _f64p]),
            "orc3_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int64, _f64p, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _f64p]),
            "orc3_destroy": (None, [vp]),
            "orc3_set_move_size": (ctypes.c_int, [vp, ctypes.c_double]),
            "orc3_set_balance": (None, [vp, ctypes.c_int, ctypes.c_int]),
            "orc3_sweep_draws": (None, [ctypes.c_uint64, ctypes.c_uint32, _f64p, _i32p, _i32p, _f64p]),
            "orc3_cell_draws": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _f64p]),
            "orc3_sweep": (ctypes.c_int, [vp, ctypes.c_int64]),
            "orc3_shift": (ctypes.c_int, [vp]),
            "orc3_subsweep": (None, [vp, ctypes.c_uint32, ctypes.c_int]),
            "orc3_info": (None, [vp, _i32p, _f64p, _u64p, _u64p]),
            "orc3_counters": (None, [vp, _u64p]),
            "orc3_origin": (None, [vp, _f64p]),
            "orc3_state": (None, [vp, _f64p, _u8p]),
            "orc3_positions": (None, [vp, _f64p]),
            "orc3_histogram": (None, [vp, ctypes.c_int, ctypes.c_double, _u64p]),
            "orc3_local_overlaps": (ctypes.c_int, [vp]),
            "orc3_bruteforce_close_pairs": (ctypes.c_int64, [_f64p, ctypes.c_int64, _f64p, ctypes.c_double]),
            "orc3_bruteforce_histogram": (None, [_f64p, ctypes.c_int64, _f64p, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_double, _u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def stream_words(seed, c0, c1, c2, count):
    out = np.zeros(count, dtype=np.uint32)
    lib().orc_stream_words(seed, c0, c1, c2, count, _p(out, _u32p))
    return out


def stream_bounded(seed, c0, c1, c2, rng, count):
    out = np.zeros(count, dtype=np.uint32)
    lib().orc_stream_bounded(seed, c0, c1, c2, rng, count, _p(out, _u32p))
    return out


def lemire_exhaustive(rng):
    out = np.zeros(rng, dtype=np.uint64)
    lib().orc_lemire_exhaustive(rng, _p(out, _u64p))
    return out


CELLS_SIGMA, CELLS_SQRT2 = 0, 1   # grid rules: cells just wider than sigma / the paper's just below sqrt(2) sigma


def grid(Lx, Ly, sigma=1.0, cells=CELLS_SIGMA):
    mx, my = ctypes.c_int32(), ctypes.c_int32()
    wx, wy = ctypes.c_double(), ctypes.c_double()
    err = lib().orc_grid_rule(Lx, Ly, sigma, cells, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(wx),
                              ctypes.byref(wy))
    if err:
        raise ValueError("invalid box")
    return mx.value, my.value, wx.value, wy.value


def lattice_shape(N, Lx, Ly):
    nx, ny = ctypes.c_int64(), ctypes.c_int64()
    if lib().orc_lattice_shape(N, Lx, Ly, ctypes.byref(nx), ctypes.byref(ny)):
        raise ValueError("no lattice shape")
    return nx.value, ny.value


def lattice_positions(N, Lx, Ly, sigma, seed):
    xy = np.zeros(2 * N, dtype=np.float64)
    if lib().orc_lattice_positions(N, Lx, Ly, sigma, seed, _p(xy, _f64p)):
        raise ValueError("no lattice")
    return xy.reshape(N, 2)


def sweep_draws(seed, sweep, wx, wy):
    perm = np.zeros(4, dtype=np.int32)
    f = ctypes.c_int32()
    ds = ctypes.c_double()
    lib().orc_sweep_draws(seed, sweep, wx, wy, _p(perm, _i32p), ctypes.byref(f), ctypes.byref(ds))
    return perm, f.value, ds.value


def close_pairs(xy, Lx, Ly, rmin):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    return int(lib().orc_bruteforce_close_pairs(_p(xy, _f64p), xy.size // 2, Lx, Ly, rmin))


def bruteforce_histogram(xy, Lx, Ly, sigma, nbins, dr):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    h = np.zeros(nbins, dtype=np.uint64)
    lib().orc_bruteforce_histogram(_p(xy, _f64p), xy.size // 2, Lx, Ly, sigma, nbins, dr, _p(h, _u64p))
    return h


def bruteforce_psi6(xy, Lx, Ly, rcut):
    """psi_6 sums and per-disk values by brute force over all pairs and the
    3x3 periodic images of global coordinates."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    out = np.zeros(4, dtype=np.float64)
    psi = np.zeros(xy.size, dtype=np.float64)
    lib().orc_bruteforce_psi6(_p(xy, _f64p), xy.size // 2, Lx, Ly, rcut, _p(out, _f64p), _p(psi, _f64p))
    return out, psi.reshape(-1, 2)


def displacements(seed, sweep, Q, t, precision, ncells):
    """Accepted (u,v) of trial t for cells 0..ncells-1 (unit-disk directions)."""
    uv = np.zeros(2 * ncells, dtype=np.float64)
    lib().orc_displacements(seed, sweep, Q, t, precision, ncells, _p(uv, _f64p))
    return uv.reshape(ncells, 2)


def shuffles(seed, sweep, Q, n, ncells, precision=FP64):
    """Shuffle orders of n slots for cells 0..ncells-1 (perm[j] = old slot now at j)."""
    out = np.zeros(4 * ncells, dtype=np.int32)
    lib().orc_shuffles(seed, sweep, Q, n, precision, ncells, _p(out, _i32p))
    return out.reshape(ncells, 4)[:, :n]


def lemire21_exhaustive(rng):
    out = np.zeros(rng, dtype=np.uint64)
    lib().orc_lemire21_exhaustive(rng, _p(out, _u64p))
    return out


def fields21(words):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    f = np.zeros(6, dtype=np.uint32)
    lib().orc_fields21(_p(w, _u32p), _p(f, _u32p))
    return f


def decode_perm(n, k):
    out = np.zeros(4, dtype=np.int32)
    lib().orc_decode_perm(n, k, _p(out, _i32p))
    return out[:n]


def visit_sequence(n, nsel):
    out = np.zeros(nsel, dtype=np.int32)
    lib().orc_visit_sequence(n, nsel, _p(out, _i32p))
    return out


def squared_bin_edges(sigma, dr, nbins):
    E = np.zeros(nbins + 1, dtype=np.float64)
    lib().orc_edges2(sigma, dr, nbins, _p(E, _f64p))
    return E


def set_threads(n):
    return int(lib().orc_set_threads(n))


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with oracle error %d" % (what, code))
        self.code = code


class System:
    """One hard-disk system advanced by the oracle."""

    def __init__(self, N, Lx, Ly, sigma=1.0, d=0.1, nselect=4, seed=1, precision=FP64, xy=None, cells=CELLS_SIGMA):
        self._h = ctypes.c_void_p()
        L = lib()
        mode = precision + 256 * cells
        if xy is None:
            err = L.orc_create(ctypes.byref(self._h), N, Lx, Ly, sigma, d, nselect, seed, mode)
        else:
            xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
            err = L.orc_create_from(ctypes.byref(self._h), N, Lx, Ly, sigma, d, nselect, seed, mode,
                                    _p(xy, _f64p))
        if err:
            raise OracleError(err, "create")
        self.N, self.Lx, self.Ly, self.sigma = N, Lx, Ly, sigma
        self.precision = precision
        self.mx, self.my, self.wx, self.wy, _, _ = self.info()
        self.C = self.mx * self.my

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_destroy(h)
            self._h = None

    def info(self):
        mx, my = ctypes.c_int32(), ctypes.c_int32()
        wx, wy = ctypes.c_double(), ctypes.c_double()
        s, k = ctypes.c_uint64(), ctypes.c_uint64()
        lib().orc_info(self._h, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(wx), ctypes.byref(wy),
                       ctypes.byref(s), ctypes.byref(k))
        return mx.value, my.value, wx.value, wy.value, s.value, k.value

    @property
    def sweeps_done(self):
        return self.info()[4]

    def sweep(self, n=1):
        err = lib().orc_sweep(self._h, n)
        if err:
            raise OracleError(err, "sweep")

    def shift(self):
        err = lib().orc_shift(self._h)
        if err:
            raise OracleError(err, "shift")

    def subsweep(self, sweep_index, Q):
        lib().orc_subsweep(self._h, sweep_index, Q)

    def set_move_size(self, d):
        if lib().orc_set_move_size(self._h, d):
            raise ValueError("bad move size")

    def set_balance(self, shuffle_particles=True, shuffle_sets=True):
        lib().orc_set_balance(self._h, int(shuffle_particles), int(shuffle_sets))

    def set_allow_leave(self, allow=True):
        """Negative control of Sec. 2.4 item 1 (either mode, serial order):
        moves that leave the cell are made instead of rejected."""
        if lib().orc_set_allow_leave(self._h, int(allow)):
            raise ValueError("allow_leave failed")

    def set_strips(self, nstrips):
        """Spatial decomposition with inactive bands (Sec. 6): the first cell
        row of each of nstrips strips makes no trial moves (0 = none)."""
        if lib().orc_set_strips(self._h, int(nstrips)):
            raise ValueError("need my >= 2 nstrips")

    def strip_rows(self, nstrips):
        """[(first row, end row) of strip k for k < nstrips]."""
        r = [lib().orc_strip_start(self.my, nstrips, k) for k in range(nstrips)] + [self.my]
        return [(r[k], r[k + 1]) for k in range(nstrips)]

    def sweep_phase(self, phase):
        """Phase 0: the sub-sweeps of the next sweep; phase 1: its grid shift."""
        err = lib().orc_sweep_phase(self._h, int(phase))
        if err:
            raise OracleError(err, "sweep_phase")

    def get_row(self, cy):
        """Cell row cy: (local[mx, 4, 2], counts[mx])."""
        loc = np.zeros(self.mx * 8, dtype=np.float64)
        cnt = np.zeros(self.mx, dtype=np.uint8)
        lib().orc_get_row(self._h, int(cy), _p(loc, _f64p), _p(cnt, _u8p))
        return loc.reshape(self.mx, 4, 2), cnt

    def set_row(self, cy, local, counts):
        loc = np.ascontiguousarray(local, dtype=np.float64).reshape(-1)
        cnt = np.ascontiguousarray(counts, dtype=np.uint8)
        lib().orc_set_row(self._h, int(cy), _p(loc, _f64p), _p(cnt, _u8p))

    def counters(self):
        out = np.zeros(4, dtype=np.uint64)
        lib().orc_counters(self._h, _p(out, _u64p))
        return out

    def origin(self):
        out = np.zeros(2, dtype=np.float64)
        lib().orc_origin(self._h, _p(out, _f64p))
        return out

    def state(self):
        """(local[C,4,2] float64, counts[C] uint8) in canonical cell order c = cy*mx + cx."""
        loc = np.zeros(self.C * 8, dtype=np.float64)
        cnt = np.zeros(self.C, dtype=np.uint8)
        lib().orc_state(self._h, _p(loc, _f64p), _p(cnt, _u8p))
        return loc.reshape(self.C, 4, 2), cnt

    def positions(self):
        xy = np.zeros(2 * self.N, dtype=np.float64)
        lib().orc_positions(self._h, _p(xy, _f64p))
        return xy.reshape(self.N, 2)

    def box(self):
        """Periodic box of the mode's geometry (binary32 cell widths in FP32 mode)."""
        if self.precision == FP64:
            return self.Lx, self.Ly
        return self.mx * float(np.float32(self.wx)), self.my * float(np.float32(self.wy))

    def histogram(self, nbins=200, dr=pressure.DR):
        h = np.zeros(nbins, dtype=np.uint64)
        lib().orc_histogram(self._h, nbins, dr * self.sigma, _p(h, _u64p))
        return h

    def psi6(self, rcut=None, per_disk=False):
        """Sums (re, im, |.|, neighbours) of psi_6 over the disks; with
        per_disk, also psi_6 of every slot, shape (mx*my, 4, 2)."""
        rcut = 1.4 * self.sigma if rcut is None else rcut
        out = np.zeros(4, dtype=np.float64)
        if per_disk:
            psi = np.zeros(8 * self.mx * self.my, dtype=np.float64)
            lib().orc_psi6(self._h, rcut, _p(out, _f64p), _p(psi, _f64p))
            return out, psi.reshape(-1, 4, 2)
        lib().orc_psi6(self._h, rcut, _p(out, _f64p), None)
        return out

    def local_overlaps(self):
        return int(lib().orc_local_overlaps(self._h))


# ---------------------------------------------------------------------------
# Three dimensions: hard spheres (eight checkerboard sets)
# ---------------------------------------------------------------------------
def _box3(L):
    return np.ascontiguousarray(L, dtype=np.float64).reshape(3)


def grid3(L, sigma=1.0):
    """(m[3], w[3]) of the 3-d cell grid; ValueError if the box is invalid."""
    Lb = _box3(L)
    m = np.zeros(3, dtype=np.int32)
    w = np.zeros(3, dtype=np.float64)
    if lib().orc3_grid(_p(Lb, _f64p), sigma, _p(m, _i32p), _p(w, _f64p)):
        raise ValueError("invalid box")
    return m, w


def lattice3_positions(N, L, sigma, seed):
    Lb = _box3(L)
    xyz = np.zeros(3 * N, dtype=np.float64)
    if lib().orc3_lattice_positions(N, _p(Lb, _f64p), sigma, seed, _p(xyz, _f64p)):
        raise ValueError("no fcc lattice for N = %d" % N)
    return xyz.reshape(N, 3)


def decode_perm8(n, k):
    out = np.zeros(8, dtype=np.int32)
    lib().orc3_decode_perm(n, k, _p(out, _i32p))
    return out[:n]


def sweep_draws3(seed, sweep, w):
    wb = _box3(w)
    perm = np.zeros(8, dtype=np.int32)
    f = ctypes.c_int32()
    ds = ctypes.c_double()
    lib().orc3_sweep_draws(seed, sweep, _p(wb, _f64p), _p(perm, _i32p), ctypes.byref(f), ctypes.byref(ds))
    return perm, f.value, ds.value


def cell_draws3(seed, sweep, cell, Q, n, nsel, shuffle=True, precision=FP64):
    """(perm[:n], uvw[nsel, 3]) of one 3-d cell update."""
    perm = np.zeros(8, dtype=np.int32)
    uvw = np.zeros(3 * nsel, dtype=np.float64)
    lib().orc3_cell_draws(seed, sweep, cell, Q, n, int(shuffle), nsel, precision, _p(perm, _i32p),
                          _p(uvw, _f64p))
    return perm[:n], uvw.reshape(nsel, 3)


def close_pairs3(xyz, L, rmin):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    Lb = _box3(L)
    return int(lib().orc3_bruteforce_close_pairs(_p(xyz, _f64p), xyz.size // 3, _p(Lb, _f64p), rmin))


def bruteforce_histogram3(xyz, L, sigma, nbins, dr):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    Lb = _box3(L)
    h = np.zeros(nbins, dtype=np.uint64)
    lib().orc3_bruteforce_histogram(_p(xyz, _f64p), xyz.size // 3, _p(Lb, _f64p), sigma, nbins, dr, _p(h, _u64p))
    return h


class System3:
    """One hard-sphere system advanced by the oracle (three dimensions)."""

    def __init__(self, N, L, sigma=1.0, d=0.1, nselect=4, seed=1, precision=FP64, xyz=None):
        self._h = ctypes.c_void_p()
        self.L = _box3(L).copy()
        arg = None
        if xyz is not None:
            xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
            arg = _p(xyz, _f64p)
        err = lib().orc3_create(ctypes.byref(self._h), N, _p(self.L, _f64p), sigma, d, nselect, seed,
                                precision, arg)
        if err:
            raise OracleError(err, "create")
        self.N, self.sigma, self.precision = N, sigma, precision
        self.m, self.w, _, _ = self.info()
        self.C = int(np.prod(self.m.astype(np.int64)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc3_destroy(h)
            self._h = None

    def info(self):
        m = np.zeros(3, dtype=np.int32)
        w = np.zeros(3, dtype=np.float64)
        s, k = ctypes.c_uint64(), ctypes.c_uint64()
        lib().orc3_info(self._h, _p(m, _i32p), _p(w, _f64p), ctypes.byref(s), ctypes.byref(k))
        return m, w, s.value, k.value

    def sweep(self, n=1):
        err = lib().orc3_sweep(self._h, n)
        if err:
            raise OracleError(err, "sweep")

    def shift(self):
        err = lib().orc3_shift(self._h)
        if err:
            raise OracleError(err, "shift")

    def subsweep(self, sweep_index, Q):
        lib().orc3_subsweep(self._h, sweep_index, Q)

    def set_move_size(self, d):
        if lib().orc3_set_move_size(self._h, d):
            raise ValueError("bad move size")

    def set_balance(self, shuffle_particles=True, shuffle_sets=True):
        lib().orc3_set_balance(self._h, int(shuffle_particles), int(shuffle_sets))

    def counters(self):
        out = np.zeros(4, dtype=np.uint64)
        lib().orc3_counters(self._h, _p(out, _u64p))
        return out

    def origin(self):
        out = np.zeros(3, dtype=np.float64)
        lib().orc3_origin(self._h, _p(out, _f64p))
        return out

    def state(self):
        """(local[C,8,3] float64, counts[C] uint8), c = (cz*my + cy)*mx + cx."""
        loc = np.zeros(self.C * 24, dtype=np.float64)
        cnt = np.zeros(self.C, dtype=np.uint8)
        lib().orc3_state(self._h, _p(loc, _f64p), _p(cnt, _u8p))
        return loc.reshape(self.C, 8, 3), cnt

    def positions(self):
        xyz = np.zeros(3 * self.N, dtype=np.float64)
        lib().orc3_positions(self._h, _p(xyz, _f64p))
        return xyz.reshape(self.N, 3)

    def box(self):
        """Periodic box of the mode's geometry (binary32 cell widths in FP32 mode)."""
        if self.precision == FP64:
            return self.L.copy()
        return self.m * self.w.astype(np.float32).astype(np.float64)

    def histogram(self, nbins=200, dr=pressure.DR):
        h = np.zeros(nbins, dtype=np.uint64)
        lib().orc3_histogram(self._h, nbins, dr * self.sigma, _p(h, _u64p))
        return h

    def local_overlaps(self):
        return int(lib().orc3_local_overlaps(self._h))
