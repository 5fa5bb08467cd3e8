"""Python binding of libhdmc.so (include/hdmc.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all Monte Carlo work runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace) and the CUDA stream.
If libhdmc.so has not been built, every call raises; there is no CPU path.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HDMC_OK, HDMC_EINVAL, HDMC_ECUDA, HDMC_EOVERFLOW, HDMC_EOVERLAP, HDMC_ETIMEOUT, HDMC_ENOMEM, HDMC_ECHECK = range(8)
HDMC_BUILD_CHECK = 1
HDMC_FP64, HDMC_FP32_LOCAL = 0, 1
HDMC_CELLS_SQRT2 = 0x100
HDMC_EMPTY_SLOT = -1.0e4
HDMC_HIST_BINS = 200
HDMC_NOALLOC_MAX_BINS = 1024

_PRECISIONS = {"fp64": HDMC_FP64, "fp32": HDMC_FP32_LOCAL, "fp32_local": HDMC_FP32_LOCAL,
               HDMC_FP64: HDMC_FP64, HDMC_FP32_LOCAL: HDMC_FP32_LOCAL}

_lib = None
_vp = ctypes.c_void_p
_f64p = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)

# name -> (restype, argtypes), as declared in include/hdmc.h
SIGNATURES = {
    "hdmc_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int]),
    "hdmc_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                   _vp, ctypes.c_size_t, _vp]),
    "hdmc_set_positions": (ctypes.c_int, [_vp, _f64p]),
    "hdmc_sweep": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "hdmc_shift": (ctypes.c_int, [_vp]),
    "hdmc_sample": (ctypes.c_int, [_vp]),
    "hdmc_pressure": (ctypes.c_int, [_vp, _f64p, _f64p, _u64p, _i64p]),
    "hdmc_positions": (ctypes.c_int, [_vp, _f64p, _i32p]),
    "hdmc_psi6": (ctypes.c_int, [_vp, ctypes.c_double, _f64p, _f64p]),
    "hdmc_get_state": (ctypes.c_int, [_vp, _f64p, _u8p]),
    "hdmc_set_state": (ctypes.c_int, [_vp, _f64p, _u8p, _f64p, ctypes.c_uint64, ctypes.c_uint64]),
    "hdmc_snapshot_bytes": (ctypes.c_size_t, [_vp]),
    "hdmc_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc_counters": (ctypes.c_int, [_vp, _u64p]),
    "hdmc_info": (ctypes.c_int, [_vp, _i32p, _i32p, _f64p, _f64p, _u64p, _u64p, _f64p]),
    "hdmc_set_move_size": (ctypes.c_int, [_vp, ctypes.c_double]),
    "hdmc_tune_move_size": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _f64p]),
    "hdmc_set_balance": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "hdmc_set_stream": (ctypes.c_int, [_vp, _vp]),
    "hdmc_sync": (ctypes.c_int, [_vp]),
    "hdmc_profile_sweeps": (ctypes.c_int, [_vp, ctypes.c_int64, _f64p, _f64p, _f64p]),
    "hdmc_profile_stages": (ctypes.c_int, [_vp, ctypes.c_int64, _f64p, _f64p]),
    "hdmc_histogram_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int32, ctypes.c_double, _u64p, _vp]),
    "hdmc_strip_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int32, ctypes.c_int32, _vp]),
    "hdmc_strip_rows": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "hdmc_strip_subsweeps": (ctypes.c_int, [_vp]),
    "hdmc_strip_shift": (ctypes.c_int, [_vp]),
    "hdmc_strip_row_bytes": (ctypes.c_size_t, [_vp]),
    "hdmc_strip_get_row": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "hdmc_strip_set_halo": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "hdmc_strip_histogram": (ctypes.c_int, [_vp, _u64p, _i64p]),
    "hdmc_pressure_fit": (ctypes.c_int, [_u64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _f64p, _f64p]),
    "hdmc_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, _i64p, _f64p, _f64p, ctypes.c_double,
                                                     ctypes.c_int]),
    "hdmc_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, _f64p, _f64p, ctypes.c_double,
                                         _f64p, _i32p, _u64p, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "hdmc_batch_sweep": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "hdmc_batch_sample": (ctypes.c_int, [_vp]),
    "hdmc_batch_pressure": (ctypes.c_int, [_vp, _f64p, _f64p, _u64p, _i64p]),
    "hdmc_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int, _f64p, _u8p]),
    "hdmc_batch_set_state": (ctypes.c_int, [_vp, ctypes.c_int, _f64p, _u8p, _f64p, ctypes.c_uint64]),
    "hdmc_batch_counters": (ctypes.c_int, [_vp, _u64p]),
    "hdmc_batch_psi6": (ctypes.c_int, [_vp, ctypes.c_double, _f64p]),
    "hdmc_batch_snapshot_bytes": (ctypes.c_size_t, [_vp]),
    "hdmc_batch_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc_batch_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc_batch_info": (ctypes.c_int, [_vp, ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _u64p, _f64p]),
    "hdmc_batch_set_nselect": (ctypes.c_int, [_vp, _i32p]),
    "hdmc_batch_set_rows": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "hdmc_batch_set_balance": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "hdmc_batch_config": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "hdmc_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int64, _i32p, _i32p]),
    "hdmc_batch_destroy": (None, [_vp]),
    "hdmc_destroy": (None, [_vp]),
    "hdmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "hdmc_build_flags": (ctypes.c_int, []),
    # three dimensions
    "hdmc3_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_int, _f64p, _vp]),
    "hdmc3_sweep": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "hdmc3_shift": (ctypes.c_int, [_vp]),
    "hdmc3_subsweep": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_int]),
    "hdmc3_sample": (ctypes.c_int, [_vp]),
    "hdmc3_pressure": (ctypes.c_int, [_vp, _f64p, _f64p, _u64p, _i64p]),
    "hdmc3_positions": (ctypes.c_int, [_vp, _f64p]),
    "hdmc3_get_state": (ctypes.c_int, [_vp, _f64p, _u8p]),
    "hdmc3_counters": (ctypes.c_int, [_vp, _u64p]),
    "hdmc3_info": (ctypes.c_int, [_vp, _i32p, _f64p, _f64p, _u64p, _u64p]),
    "hdmc3_set_move_size": (ctypes.c_int, [_vp, ctypes.c_double]),
    "hdmc3_set_balance": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "hdmc3_sync": (ctypes.c_int, [_vp]),
    "hdmc3_snapshot_bytes": (ctypes.c_size_t, [_vp]),
    "hdmc3_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc3_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hdmc3_profile_sweeps": (ctypes.c_int, [_vp, ctypes.c_int64, _f64p, _f64p]),
    "hdmc3_profile_stages": (ctypes.c_int, [_vp, ctypes.c_int64, _f64p, _f64p]),
    "hdmc3_destroy": (None, [_vp]),
}


class HDMCError(RuntimeError):
    def __init__(self, code, where):
        msg = "%s: %s (code %d)" % (where, hdmc_strerror(code) if _lib is not None else "error", code)
        super().__init__(msg)
        self.code = code


def library_path():
    return _build.LIB


def lib():
    """The loaded libhdmc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libhdmc.so is not built (%s); run __graft_entry__.build() first" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code, where):
    if code != HDMC_OK:
        raise HDMCError(code, where)


def _p(a, t):
    return a.ctypes.data_as(t)


def _precision(p):
    """HDMC_FP64 / HDMC_FP32_LOCAL from a name or value; an int may carry HDMC_CELLS_SQRT2."""
    if isinstance(p, int) and (p & ~0xFF) == HDMC_CELLS_SQRT2 and (p & 0xFF) in _PRECISIONS:
        return p
    try:
        return _PRECISIONS[p]
    except KeyError:
        raise ValueError("precision must be 'fp64' or 'fp32'") from None


def with_cells(precision, cells):
    """precision for the library calls with cell rule cells ('sigma' or 'sqrt2')."""
    if cells not in ("sigma", "sqrt2"):
        raise ValueError("cells must be 'sigma' or 'sqrt2'")
    return _precision(precision) | (HDMC_CELLS_SQRT2 if cells == "sqrt2" else 0)


# ---- one Python function per C entry point ----------------------------------------

def hdmc_strerror(code):
    return lib().hdmc_strerror(code).decode()


def hdmc_build_flags():
    return int(lib().hdmc_build_flags())


def hdmc_workspace_bytes(N, Lx, Ly, sigma, precision):
    return int(lib().hdmc_workspace_bytes(N, Lx, Ly, sigma, _precision(precision)))


def hdmc_create(N, Lx, Ly, sigma, d, nselect, seed, precision, dev_workspace=None, workspace_bytes=0,
                stream=None):
    h = _vp()
    _check(lib().hdmc_create(ctypes.byref(h), N, Lx, Ly, sigma, d, nselect, seed & 0xFFFFFFFFFFFFFFFF,
                             _precision(precision), dev_workspace, workspace_bytes, stream), "hdmc_create")
    return h


def hdmc_set_positions(h, xy):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    _check(lib().hdmc_set_positions(h, _p(xy, _f64p)), "hdmc_set_positions")


def hdmc_sweep(h, n):
    _check(lib().hdmc_sweep(h, n), "hdmc_sweep")


def hdmc_shift(h):
    _check(lib().hdmc_shift(h), "hdmc_shift")


def hdmc_sample(h):
    _check(lib().hdmc_sample(h), "hdmc_sample")


def hdmc_pressure(h):
    """Returns (betaP_over_rho, g_contact, hist[200] uint64, n_samples)."""
    bp, g0 = ctypes.c_double(), ctypes.c_double()
    ns = ctypes.c_int64()
    hist = np.zeros(HDMC_HIST_BINS, dtype=np.uint64)
    _check(lib().hdmc_pressure(h, ctypes.byref(bp), ctypes.byref(g0), _p(hist, _u64p), ctypes.byref(ns)),
           "hdmc_pressure")
    return bp.value, g0.value, hist, ns.value


def hdmc_positions(h, N):
    xy = np.zeros(2 * N, dtype=np.float64)
    cell = np.zeros(N, dtype=np.int32)
    _check(lib().hdmc_positions(h, _p(xy, _f64p), _p(cell, _i32p)), "hdmc_positions")
    return xy.reshape(N, 2), cell


def hdmc_psi6(h, r_cut, C=None):
    """(mean psi_6 as a complex number, mean |psi_6|, mean neighbours), and
    psi_6 of every slot, shape (C, 4, 2), when C (cells) is given."""
    out = np.zeros(4, dtype=np.float64)
    if C is None:
        _check(lib().hdmc_psi6(h, r_cut, _p(out, _f64p), None), "hdmc_psi6")
        return complex(out[0], out[1]), out[2], out[3]
    psi = np.zeros(8 * C, dtype=np.float64)
    _check(lib().hdmc_psi6(h, r_cut, _p(out, _f64p), _p(psi, _f64p)), "hdmc_psi6")
    return complex(out[0], out[1]), out[2], out[3], psi.reshape(C, 4, 2)


def hdmc_get_state(h, C):
    loc = np.zeros(8 * C, dtype=np.float64)
    cnt = np.zeros(C, dtype=np.uint8)
    _check(lib().hdmc_get_state(h, _p(loc, _f64p), _p(cnt, _u8p)), "hdmc_get_state")
    return loc.reshape(C, 4, 2), cnt


def hdmc_set_state(h, local, counts, origin, sweeps_done, shifts_done):
    loc = np.ascontiguousarray(local, dtype=np.float64).reshape(-1)
    cnt = np.ascontiguousarray(counts, dtype=np.uint8)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    _check(lib().hdmc_set_state(h, _p(loc, _f64p), _p(cnt, _u8p), _p(org, _f64p), sweeps_done, shifts_done),
           "hdmc_set_state")


def _host_buffer(buf):
    """(address, size in bytes) of a contiguous host buffer: a numpy array or
    a CPU torch tensor (pinned or not)."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("snapshot buffer must be contiguous")
        return buf.ctypes.data, buf.nbytes
    if buf.device.type != "cpu" or not buf.is_contiguous():
        raise ValueError("snapshot buffer must be a contiguous host tensor")
    return buf.data_ptr(), buf.numel() * buf.element_size()


def hdmc_snapshot_bytes(h):
    return int(lib().hdmc_snapshot_bytes(h))


def hdmc_save(h, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc_save(h, ptr, n), "hdmc_save")
    return buf


def hdmc_load(h, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc_load(h, ptr, n), "hdmc_load")


def hdmc_counters(h):
    out = np.zeros(4, dtype=np.uint64)
    _check(lib().hdmc_counters(h, _p(out, _u64p)), "hdmc_counters")
    return out


def hdmc_info(h):
    mx, my = ctypes.c_int32(), ctypes.c_int32()
    wx, wy = ctypes.c_double(), ctypes.c_double()
    sw, sh = ctypes.c_uint64(), ctypes.c_uint64()
    org = np.zeros(2, dtype=np.float64)
    _check(lib().hdmc_info(h, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(wx), ctypes.byref(wy),
                           ctypes.byref(sw), ctypes.byref(sh), _p(org, _f64p)), "hdmc_info")
    return {"mx": mx.value, "my": my.value, "wx": wx.value, "wy": wy.value, "sweeps_done": sw.value,
            "shifts_done": sh.value, "origin": org}


def hdmc_set_move_size(h, d):
    _check(lib().hdmc_set_move_size(h, d), "hdmc_set_move_size")


def hdmc_set_balance(h, shuffle_particles, shuffle_sets):
    _check(lib().hdmc_set_balance(h, int(bool(shuffle_particles)), int(bool(shuffle_sets))), "hdmc_set_balance")


def hdmc_tune_move_size(h, target, sweeps, every):
    d = ctypes.c_double()
    _check(lib().hdmc_tune_move_size(h, target, sweeps, every, ctypes.byref(d)), "hdmc_tune_move_size")
    return d.value


def hdmc_set_stream(h, stream):
    _check(lib().hdmc_set_stream(h, stream), "hdmc_set_stream")


def hdmc_sync(h):
    _check(lib().hdmc_sync(h), "hdmc_sync")


def hdmc_profile_sweeps(h, n):
    """Returns mean ms per (sub-sweep, shift, draws) launch over n directly launched sweeps."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().hdmc_profile_sweeps(h, n, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "hdmc_profile_sweeps")
    return a.value, b.value, c.value


def hdmc_profile_stages(h, n):
    """Returns mean ms per (sub-sweep, shift) launch inside recorded graphs of n sweeps of one stage each."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().hdmc_profile_stages(h, n, ctypes.byref(a), ctypes.byref(b)), "hdmc_profile_stages")
    return a.value, b.value


def hdmc_histogram_noalloc(dev_local, mx, my, wx, wy, sigma, nbins, dr, stream=None):
    """Contact histogram of a caller-owned device state (device pointer to
    8*mx*my doubles in the hdmc_get_state layout) without any device
    allocation; returns nbins uint64 counts."""
    hist = np.zeros(nbins, dtype=np.uint64)
    _check(lib().hdmc_histogram_noalloc(dev_local, mx, my, wx, wy, sigma, nbins, dr, _p(hist, _u64p), stream),
           "hdmc_histogram_noalloc")
    return hist


def hdmc_strip_create(N, Lx, Ly, sigma, d, nselect, seed, precision, nstrips, strip, stream=None):
    h = _vp()
    _check(lib().hdmc_strip_create(ctypes.byref(h), N, Lx, Ly, sigma, d, nselect, seed & 0xFFFFFFFFFFFFFFFF,
                                   _precision(precision), nstrips, strip, stream), "hdmc_strip_create")
    return h


def hdmc_strip_rows(h):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().hdmc_strip_rows(h, ctypes.byref(a), ctypes.byref(b)), "hdmc_strip_rows")
    return a.value, b.value


def hdmc_strip_subsweeps(h):
    _check(lib().hdmc_strip_subsweeps(h), "hdmc_strip_subsweeps")


def hdmc_strip_shift(h):
    _check(lib().hdmc_strip_shift(h), "hdmc_strip_shift")


def hdmc_strip_row_bytes(h):
    return int(lib().hdmc_strip_row_bytes(h))


def hdmc_strip_get_row(h, which, buf_ptr):
    _check(lib().hdmc_strip_get_row(h, which, buf_ptr), "hdmc_strip_get_row")


def hdmc_strip_set_halo(h, which, buf_ptr):
    _check(lib().hdmc_strip_set_halo(h, which, buf_ptr), "hdmc_strip_set_halo")


def hdmc_strip_histogram(h):
    hist = np.zeros(HDMC_HIST_BINS, dtype=np.uint64)
    ns = ctypes.c_int64()
    _check(lib().hdmc_strip_histogram(h, _p(hist, _u64p), ctypes.byref(ns)), "hdmc_strip_histogram")
    return hist, ns.value


def hdmc_pressure_fit(hist, n_samples, N, Lx, Ly, sigma=1.0):
    """(beta P / rho, g(sigma+)) of a contact histogram (Sec. 4)."""
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    bp, g0 = ctypes.c_double(), ctypes.c_double()
    _check(lib().hdmc_pressure_fit(_p(h, _u64p), n_samples, N, Lx, Ly, sigma, ctypes.byref(bp), ctypes.byref(g0)),
           "hdmc_pressure_fit")
    return bp.value, g0.value


def hdmc_destroy(h):
    if h is not None and h.value:
        lib().hdmc_destroy(h)


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def hdmc_batch_workspace_bytes(N, Lx, Ly, sigma, precision):
    N, Lx, Ly = _arr(N, np.int64), _arr(Lx, np.float64), _arr(Ly, np.float64)
    return int(lib().hdmc_batch_workspace_bytes(len(N), _p(N, _i64p), _p(Lx, _f64p), _p(Ly, _f64p), sigma,
                                                _precision(precision)))


def hdmc_batch_create(N, Lx, Ly, sigma, d, nselect, seeds, precision, dev_workspace=None, workspace_bytes=0,
                      stream=None):
    N, Lx, Ly, d = _arr(N, np.int64), _arr(Lx, np.float64), _arr(Ly, np.float64), _arr(d, np.float64)
    ns = None if nselect is None else _arr(nselect, np.int32)
    sd = _arr([s & 0xFFFFFFFFFFFFFFFF for s in seeds], np.uint64)
    b = _vp()
    _check(lib().hdmc_batch_create(ctypes.byref(b), len(N), _p(N, _i64p), _p(Lx, _f64p), _p(Ly, _f64p), sigma,
                                   _p(d, _f64p), None if ns is None else _p(ns, _i32p), _p(sd, _u64p),
                                   _precision(precision), dev_workspace, workspace_bytes, stream), "hdmc_batch_create")
    return b


def hdmc_batch_sweep(b, n):
    _check(lib().hdmc_batch_sweep(b, n), "hdmc_batch_sweep")


def hdmc_batch_sample(b):
    _check(lib().hdmc_batch_sample(b), "hdmc_batch_sample")


def hdmc_batch_pressure(b, R):
    """Returns (betaP_over_rho[R], g_contact[R], hist[R, 200], n_samples)."""
    bp, g0 = np.zeros(R), np.zeros(R)
    hist = np.zeros(R * HDMC_HIST_BINS, dtype=np.uint64)
    ns = ctypes.c_int64()
    _check(lib().hdmc_batch_pressure(b, _p(bp, _f64p), _p(g0, _f64p), _p(hist, _u64p), ctypes.byref(ns)),
           "hdmc_batch_pressure")
    return bp, g0, hist.reshape(R, HDMC_HIST_BINS), ns.value


def hdmc_batch_get_state(b, r, C):
    loc = np.zeros(8 * C, dtype=np.float64)
    cnt = np.zeros(C, dtype=np.uint8)
    _check(lib().hdmc_batch_get_state(b, r, _p(loc, _f64p), _p(cnt, _u8p)), "hdmc_batch_get_state")
    return loc.reshape(C, 4, 2), cnt


def hdmc_batch_set_state(b, r, local, counts, origin, sweeps_done):
    loc = np.ascontiguousarray(local, dtype=np.float64).reshape(-1)
    cnt = np.ascontiguousarray(counts, dtype=np.uint8)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    _check(lib().hdmc_batch_set_state(b, r, _p(loc, _f64p), _p(cnt, _u8p), _p(org, _f64p), sweeps_done),
           "hdmc_batch_set_state")


def hdmc_batch_counters(b, R):
    out = np.zeros(4 * R, dtype=np.uint64)
    _check(lib().hdmc_batch_counters(b, _p(out, _u64p)), "hdmc_batch_counters")
    return out.reshape(R, 4)


def hdmc_batch_info(b, r):
    mx, my = ctypes.c_int32(), ctypes.c_int32()
    wx, wy = ctypes.c_double(), ctypes.c_double()
    sw = ctypes.c_uint64()
    org = np.zeros(2, dtype=np.float64)
    _check(lib().hdmc_batch_info(b, r, ctypes.byref(mx), ctypes.byref(my), ctypes.byref(wx), ctypes.byref(wy),
                                 ctypes.byref(sw), _p(org, _f64p)), "hdmc_batch_info")
    return {"mx": mx.value, "my": my.value, "wx": wx.value, "wy": wy.value, "sweeps_done": sw.value,
            "origin": org}


def hdmc_batch_set_nselect(b, nselect):
    ns = _arr(nselect, np.int32)
    _check(lib().hdmc_batch_set_nselect(b, _p(ns, _i32p)), "hdmc_batch_set_nselect")


def hdmc_batch_psi6(b, r_cut, R):
    out = np.zeros(4 * R, dtype=np.float64)
    _check(lib().hdmc_batch_psi6(b, r_cut, _p(out, _f64p)), "hdmc_batch_psi6")
    out = out.reshape(R, 4)
    return out[:, 0] + 1j * out[:, 1], out[:, 2], out[:, 3]


def hdmc_batch_snapshot_bytes(b):
    return int(lib().hdmc_batch_snapshot_bytes(b))


def hdmc_batch_save(b, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc_batch_save(b, ptr, n), "hdmc_batch_save")
    return buf


def hdmc_batch_load(b, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc_batch_load(b, ptr, n), "hdmc_batch_load")


def hdmc_batch_set_rows(b, rows):
    _check(lib().hdmc_batch_set_rows(b, rows), "hdmc_batch_set_rows")


def hdmc_batch_set_balance(b, shuffle_particles, shuffle_sets):
    p = np.ascontiguousarray([int(bool(v)) for v in shuffle_particles], dtype=np.int32)
    q = np.ascontiguousarray([int(bool(v)) for v in shuffle_sets], dtype=np.int32)
    _check(lib().hdmc_batch_set_balance(b, _p(p, _i32p), _p(q, _i32p)), "hdmc_batch_set_balance")


def hdmc_batch_config(b, R):
    rows = ctypes.c_int32()
    ns = np.zeros(R, dtype=np.int32)
    _check(lib().hdmc_batch_config(b, ctypes.byref(rows), _p(ns, _i32p)), "hdmc_batch_config")
    return rows.value, ns


def hdmc_batch_autotune(b, sweeps):
    rows, nm = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().hdmc_batch_autotune(b, sweeps, ctypes.byref(rows), ctypes.byref(nm)), "hdmc_batch_autotune")
    return rows.value, nm.value


def hdmc_batch_destroy(b):
    if b is not None and b.value:
        lib().hdmc_batch_destroy(b)


# ---- convenience wrappers ----------------------------------------------------------

class System:
    """One hard-disk system on the current CUDA device.

    The device workspace is a torch uint8 tensor (PyTorch's caching allocator
    owns the memory) and work goes to torch's current stream unless a stream
    is given.  If xy is given, the lattice start is replaced by those global
    positions.
    """

    def __init__(self, N, Lx, Ly, sigma=1.0, d=0.1, nselect=4, seed=1, precision="fp32", xy=None,
                 stream=None, device=None, cells="sigma"):
        import torch

        self.N, self.Lx, self.Ly, self.sigma = N, Lx, Ly, sigma
        self.precision = _precision(precision) & 0xFF
        mode = with_cells(self.precision, cells)   # precision argument with the cell rule
        nbytes = hdmc_workspace_bytes(N, Lx, Ly, sigma, mode)
        if nbytes == 0:
            raise HDMCError(HDMC_EINVAL, "hdmc_workspace_bytes")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self._ws.data_ptr()
        ptr = (base + 255) // 256 * 256
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        self._stream = stream
        self.h = None
        self.h = hdmc_create(N, Lx, Ly, sigma, d, nselect, seed, mode, ptr, nbytes, stream)
        info = hdmc_info(self.h)
        self.mx, self.my, self.wx, self.wy = info["mx"], info["my"], info["wx"], info["wy"]
        self.C = self.mx * self.my
        if xy is not None:
            hdmc_set_positions(self.h, xy)

    def close(self):
        if getattr(self, "h", None) is not None:
            hdmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        hdmc_sweep(self.h, n)

    def shift(self):
        hdmc_shift(self.h)

    def sample(self):
        hdmc_sample(self.h)

    def pressure(self):
        return hdmc_pressure(self.h)

    def positions(self):
        return hdmc_positions(self.h, self.N)[0]

    def state(self):
        return hdmc_get_state(self.h, self.C)

    def set_state(self, local, counts, origin, sweeps_done, shifts_done):
        hdmc_set_state(self.h, local, counts, origin, sweeps_done, shifts_done)

    def counters(self):
        return hdmc_counters(self.h)

    def psi6(self, r_cut=1.4, per_disk=False):
        """Orientational order: (mean psi_6, mean |psi_6|, mean neighbours
        [, psi_6 per slot]); r_cut in the units of the box."""
        return hdmc_psi6(self.h, r_cut, self.C if per_disk else None)

    def snapshot_bytes(self):
        return hdmc_snapshot_bytes(self.h)

    def save(self, buf=None):
        """Snapshot into buf (numpy uint8 array or host tensor, e.g. pinned);
        a new numpy array when buf is None.  Returns the buffer."""
        if buf is None:
            buf = np.empty(self.snapshot_bytes(), dtype=np.uint8)
        return hdmc_save(self.h, buf)

    def load(self, buf):
        hdmc_load(self.h, buf)

    def info(self):
        return hdmc_info(self.h)

    def origin(self):
        return hdmc_info(self.h)["origin"]

    def set_move_size(self, d):
        hdmc_set_move_size(self.h, d)

    def set_balance(self, shuffle_particles=True, shuffle_sets=True):
        """Table 1 negative controls (both True = the method)."""
        hdmc_set_balance(self.h, shuffle_particles, shuffle_sets)

    def tune_move_size(self, target=0.30, sweeps=1000, every=100):
        """Pre-run that sets d for the target acceptance ratio; returns d."""
        return hdmc_tune_move_size(self.h, target, sweeps, every)

    def sync(self):
        hdmc_sync(self.h)

    def box(self):
        if self.precision == HDMC_FP64:
            return self.Lx, self.Ly
        return self.mx * float(np.float32(self.wx)), self.my * float(np.float32(self.wy))


class Batch:
    """R independent systems advanced together (one launch per stage for all).

    replicas: list of objects with N, Lx, Ly, d, nselect, seed attributes
    (e.g. workloads.Workload).  Workspace and stream from PyTorch as in System.
    """

    def __init__(self, replicas, sigma=1.0, precision="fp32", stream=None, device=None, cells="sigma"):
        import torch

        self.R = len(replicas)
        self.N = [int(w.N) for w in replicas]
        self.precision = _precision(precision) & 0xFF
        mode = with_cells(self.precision, cells)
        Lx = [w.Lx for w in replicas]
        Ly = [w.Ly for w in replicas]
        nbytes = hdmc_batch_workspace_bytes(self.N, Lx, Ly, sigma, mode)
        if nbytes == 0:
            raise HDMCError(HDMC_EINVAL, "hdmc_batch_workspace_bytes")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        ptr = (self._ws.data_ptr() + 255) // 256 * 256
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        self.b = None
        self.b = hdmc_batch_create(self.N, Lx, Ly, sigma, [w.d for w in replicas], [w.nselect for w in replicas],
                                   [w.seed for w in replicas], mode, ptr, nbytes, stream)
        self.grids = [hdmc_batch_info(self.b, r) for r in range(self.R)]

    def close(self):
        if getattr(self, "b", None) is not None:
            hdmc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        hdmc_batch_sweep(self.b, n)

    def sample(self):
        hdmc_batch_sample(self.b)

    def pressure(self):
        return hdmc_batch_pressure(self.b, self.R)

    def state(self, r):
        g = self.grids[r]
        return hdmc_batch_get_state(self.b, r, g["mx"] * g["my"])

    def counters(self):
        return hdmc_batch_counters(self.b, self.R)

    def set_state(self, r, local, counts, origin, sweeps_done):
        hdmc_batch_set_state(self.b, r, local, counts, origin, sweeps_done)

    def origin(self, r):
        return hdmc_batch_info(self.b, r)["origin"]

    def set_rows(self, rows):
        hdmc_batch_set_rows(self.b, rows)

    def snapshot_bytes(self):
        return hdmc_batch_snapshot_bytes(self.b)

    def psi6(self, r_cut=1.4):
        """Per replica: mean psi_6 (complex), mean |psi_6|, mean neighbours."""
        return hdmc_batch_psi6(self.b, r_cut, self.R)

    def save(self, buf=None):
        """Snapshot of every replica into buf (numpy uint8 array or host
        tensor); a new numpy array when buf is None."""
        if buf is None:
            buf = np.empty(self.snapshot_bytes(), dtype=np.uint8)
        return hdmc_batch_save(self.b, buf)

    def load(self, buf):
        hdmc_batch_load(self.b, buf)

    def set_balance(self, shuffle_particles, shuffle_sets):
        """Per-replica Table 1 negative controls (sequences of R booleans)."""
        if len(shuffle_particles) != self.R or len(shuffle_sets) != self.R:
            raise ValueError("one value per replica")
        hdmc_batch_set_balance(self.b, shuffle_particles, shuffle_sets)

    def set_nselect(self, nselect):
        hdmc_batch_set_nselect(self.b, nselect)

    def config(self):
        return hdmc_batch_config(self.b, self.R)

    def autotune(self, sweeps=32):
        return hdmc_batch_autotune(self.b, sweeps)



# ---- three dimensions: hard spheres ------------------------------------------------

def hdmc3_create(N, L, sigma, d, nselect, seed, precision, xyz=None, stream=None):
    h = _vp()
    arg = None
    if xyz is not None:
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        arg = _p(xyz, _f64p)
    _check(lib().hdmc3_create(ctypes.byref(h), N, L[0], L[1], L[2], sigma, d, nselect, seed & 0xFFFFFFFFFFFFFFFF,
                              _precision(precision), arg, stream), "hdmc3_create")
    return h


def hdmc3_sweep(h, n):
    _check(lib().hdmc3_sweep(h, n), "hdmc3_sweep")


def hdmc3_shift(h):
    _check(lib().hdmc3_shift(h), "hdmc3_shift")


def hdmc3_subsweep(h, sweep, Q):
    _check(lib().hdmc3_subsweep(h, sweep, Q), "hdmc3_subsweep")


def hdmc3_sample(h):
    _check(lib().hdmc3_sample(h), "hdmc3_sample")


def hdmc3_pressure(h):
    """Returns (betaP_over_rho, g_contact, hist[200] uint64, n_samples)."""
    bp, g0 = ctypes.c_double(), ctypes.c_double()
    ns = ctypes.c_int64()
    hist = np.zeros(HDMC_HIST_BINS, dtype=np.uint64)
    _check(lib().hdmc3_pressure(h, ctypes.byref(bp), ctypes.byref(g0), _p(hist, _u64p), ctypes.byref(ns)),
           "hdmc3_pressure")
    return bp.value, g0.value, hist, ns.value


def hdmc3_positions(h, N):
    xyz = np.zeros(3 * N, dtype=np.float64)
    _check(lib().hdmc3_positions(h, _p(xyz, _f64p)), "hdmc3_positions")
    return xyz.reshape(N, 3)


def hdmc3_get_state(h, C):
    loc = np.zeros(24 * C, dtype=np.float64)
    cnt = np.zeros(C, dtype=np.uint8)
    _check(lib().hdmc3_get_state(h, _p(loc, _f64p), _p(cnt, _u8p)), "hdmc3_get_state")
    return loc.reshape(C, 8, 3), cnt


def hdmc3_counters(h):
    out = np.zeros(4, dtype=np.uint64)
    _check(lib().hdmc3_counters(h, _p(out, _u64p)), "hdmc3_counters")
    return out


def hdmc3_info(h):
    m = np.zeros(3, dtype=np.int32)
    w = np.zeros(3, dtype=np.float64)
    org = np.zeros(3, dtype=np.float64)
    sw, sh = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().hdmc3_info(h, _p(m, _i32p), _p(w, _f64p), _p(org, _f64p), ctypes.byref(sw), ctypes.byref(sh)),
           "hdmc3_info")
    return {"m": m, "w": w, "origin": org, "sweeps_done": sw.value, "shifts_done": sh.value}


def hdmc3_set_move_size(h, d):
    _check(lib().hdmc3_set_move_size(h, d), "hdmc3_set_move_size")


def hdmc3_set_balance(h, shuffle_particles, shuffle_sets):
    _check(lib().hdmc3_set_balance(h, int(bool(shuffle_particles)), int(bool(shuffle_sets))), "hdmc3_set_balance")


def hdmc3_sync(h):
    _check(lib().hdmc3_sync(h), "hdmc3_sync")


def hdmc3_snapshot_bytes(h):
    return int(lib().hdmc3_snapshot_bytes(h))


def hdmc3_save(h, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc3_save(h, ptr, n), "hdmc3_save")
    return buf


def hdmc3_load(h, buf):
    ptr, n = _host_buffer(buf)
    _check(lib().hdmc3_load(h, ptr, n), "hdmc3_load")


def hdmc3_profile_sweeps(h, n):
    """Mean ms per (sub-sweep, shift) launch over n sweeps."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().hdmc3_profile_sweeps(h, n, ctypes.byref(a), ctypes.byref(b)), "hdmc3_profile_sweeps")
    return a.value, b.value

def hdmc3_profile_stages(h, n):
    """Mean ms per (sub-sweep, shift) launch in runs of n sweeps of one stage each."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().hdmc3_profile_stages(h, n, ctypes.byref(a), ctypes.byref(b)), "hdmc3_profile_stages")
    return a.value, b.value


def hdmc3_destroy(h):
    if h is not None and h.value:
        lib().hdmc3_destroy(h)


class System3:
    """One hard-sphere system on the current CUDA device (work goes to torch's
    current stream unless a stream is given).  xyz: global start positions,
    else the face-centred cubic start (N = 4 q^3)."""

    def __init__(self, N, L, sigma=1.0, d=0.1, nselect=4, seed=1, precision="fp32", xyz=None, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.N, self.L, self.sigma = N, tuple(float(x) for x in L), sigma
        self.precision = _precision(precision)
        self.h = None
        self.h = hdmc3_create(N, self.L, sigma, d, nselect, seed, self.precision, xyz, stream)
        info = hdmc3_info(self.h)
        self.m, self.w = info["m"], info["w"]
        self.C = int(np.prod(self.m.astype(np.int64)))

    def close(self):
        if getattr(self, "h", None) is not None:
            hdmc3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        hdmc3_sweep(self.h, n)

    def shift(self):
        hdmc3_shift(self.h)

    def subsweep(self, sweep, Q):
        hdmc3_subsweep(self.h, sweep, Q)

    def sample(self):
        hdmc3_sample(self.h)

    def pressure(self):
        return hdmc3_pressure(self.h)

    def positions(self):
        return hdmc3_positions(self.h, self.N)

    def state(self):
        return hdmc3_get_state(self.h, self.C)

    def counters(self):
        return hdmc3_counters(self.h)

    def info(self):
        return hdmc3_info(self.h)

    def origin(self):
        return hdmc3_info(self.h)["origin"]

    def set_move_size(self, d):
        hdmc3_set_move_size(self.h, d)

    def set_balance(self, shuffle_particles=True, shuffle_sets=True):
        hdmc3_set_balance(self.h, shuffle_particles, shuffle_sets)

    def sync(self):
        hdmc3_sync(self.h)

    def snapshot_bytes(self):
        return hdmc3_snapshot_bytes(self.h)

    def save(self, buf=None):
        """Snapshot into buf (a host numpy array or CPU tensor, pinned or not;
        a new uint8 array if None); returns buf."""
        if buf is None:
            buf = np.empty(self.snapshot_bytes(), dtype=np.uint8)
        return hdmc3_save(self.h, buf)

    def load(self, buf):
        hdmc3_load(self.h, buf)

    def profile_sweeps(self, n):
        return hdmc3_profile_sweeps(self.h, n)

    def profile_stages(self, n):
        return hdmc3_profile_stages(self.h, n)

    def box(self):
        """Periodic box of the precision's geometry (binary32 cell widths in fp32)."""
        if self.precision == HDMC_FP64:
            return np.array(self.L)
        return self.m * self.w.astype(np.float32).astype(np.float64)
