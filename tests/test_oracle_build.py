"""The oracle's results do not depend on how it was compiled: a build at -O0
(every operation as written, nothing kept in registers across statements)
and the default -O2 build give bit-identical trajectories, disks and
spheres, binary64 and binary32.  This pins the floating-point contract the
parity tests rely on (no fused multiply-add unless written, no
reassociation), on whatever host compiles the oracle."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import build as oracle_build
from paper_1211_1646_gb300 import workloads as W


@pytest.fixture(scope="module")
def o0_lib(tmp_path_factory):
    oracle_build.build()
    out = str(tmp_path_factory.mktemp("oracle_o0") / "liboracle_o0.so")
    flags = [f for f in oracle_build.BASE_FLAGS if not f.startswith("-O")] + ["-O0"]
    subprocess.check_call(["gcc"] + flags + [oracle_build.SRC, "-o", out, "-lm"])
    L = ctypes.CDLL(out)
    vp = ctypes.c_void_p
    f64p = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.orc_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
    L.orc_sweep.argtypes = [vp, ctypes.c_int64]
    L.orc_state.argtypes = [vp, f64p, u8p]
    L.orc_counters.argtypes = [vp, u64p]
    L.orc_histogram.argtypes = [vp, ctypes.c_int, ctypes.c_double, u64p]
    L.orc_destroy.argtypes = [vp]
    L.orc3_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, f64p, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int, ctypes.c_uint64, ctypes.c_int, f64p]
    L.orc3_sweep.argtypes = [vp, ctypes.c_int64]
    L.orc3_state.argtypes = [vp, f64p, u8p]
    L.orc3_counters.argtypes = [vp, u64p]
    L.orc3_histogram.argtypes = [vp, ctypes.c_int, ctypes.c_double, u64p]
    L.orc3_destroy.argtypes = [vp]
    return L


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_disks_identical_at_o0(o0_lib, prec):
    w = W.n1024_phi070()
    ref = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 5, prec)
    ref.sweep(30)
    h = ctypes.c_void_p()
    assert o0_lib.orc_create(ctypes.byref(h), w.N, w.Lx, w.Ly, 1.0, w.d, 4, 5, prec) == 0
    assert o0_lib.orc_sweep(h, 30) == 0
    loc = np.zeros(ref.C * 8)
    cnt = np.zeros(ref.C, dtype=np.uint8)
    o0_lib.orc_state(h, _p(loc, ctypes.c_double), _p(cnt, ctypes.c_uint8))
    c = np.zeros(4, dtype=np.uint64)
    o0_lib.orc_counters(h, _p(c, ctypes.c_uint64))
    hist = np.zeros(200, dtype=np.uint64)
    o0_lib.orc_histogram(h, 200, 1e-4, _p(hist, ctypes.c_uint64))
    o0_lib.orc_destroy(h)
    rl, rc = ref.state()
    assert np.array_equal(loc.reshape(-1, 4, 2), rl) and np.array_equal(cnt, rc)
    assert np.array_equal(c, ref.counters())
    assert np.array_equal(hist, ref.histogram(200, 1e-4))


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_spheres_identical_at_o0(o0_lib, prec):
    w = W.spheres_n2048_phi045()
    ref = O.System3(w.N, w.L, 1.0, w.d, 4, 6, prec)
    ref.sweep(15)
    h = ctypes.c_void_p()
    L = np.array(w.L, dtype=np.float64)
    assert o0_lib.orc3_create(ctypes.byref(h), w.N, _p(L, ctypes.c_double), 1.0, w.d, 4, 6, prec, None) == 0
    assert o0_lib.orc3_sweep(h, 15) == 0
    loc = np.zeros(ref.C * 24)
    cnt = np.zeros(ref.C, dtype=np.uint8)
    o0_lib.orc3_state(h, _p(loc, ctypes.c_double), _p(cnt, ctypes.c_uint8))
    c = np.zeros(4, dtype=np.uint64)
    o0_lib.orc3_counters(h, _p(c, ctypes.c_uint64))
    hist = np.zeros(200, dtype=np.uint64)
    o0_lib.orc3_histogram(h, 200, 1e-4, _p(hist, ctypes.c_uint64))
    o0_lib.orc3_destroy(h)
    rl, rc = ref.state()
    assert np.array_equal(loc.reshape(-1, 8, 3), rl) and np.array_equal(cnt, rc)
    assert np.array_equal(c, ref.counters())
    assert np.array_equal(hist, ref.histogram(200, 1e-4))
