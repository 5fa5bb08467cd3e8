"""The C ABI (CPU only): libhdmc.so builds, loads, and exports every entry
point include/hdmc.h declares; the Python binding declares the same set.
No compute call is made here (there may be no GPU)."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hdmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hdmc3?_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1211_1646_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["hdmc_create", "hdmc_sweep", "hdmc_shift", "hdmc_pressure", "hdmc_positions", "hdmc_destroy",
              "hdmc3_create", "hdmc3_sweep", "hdmc3_shift", "hdmc3_pressure", "hdmc3_positions", "hdmc3_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_matches_header(libpath):
    from paper_1211_1646_gb300 import hdmc
    assert sorted(hdmc.SIGNATURES) == _declared()
    for n in _declared():
        assert callable(getattr(hdmc, n))
    hdmc.lib()
    assert hdmc.hdmc_strerror(hdmc.HDMC_EOVERLAP) == "overlapping disks"


def test_workspace_size_is_host_only(libpath):
    from paper_1211_1646_gb300 import hdmc, workloads
    w = workloads.n1m_phi0716()
    b32 = hdmc.hdmc_workspace_bytes(w.N, w.Lx, w.Ly, 1.0, "fp32")
    b64 = hdmc.hdmc_workspace_bytes(w.N, w.Lx, w.Ly, 1.0, "fp64")
    C = 1152 * 998
    assert 2 * C * 32 <= b32 < 2 * C * 32 + (1 << 20)
    assert 2 * C * 64 <= b64 < 2 * C * 64 + (1 << 20)
    assert hdmc.hdmc_workspace_bytes(w.N, 3.0, 3.0, 1.0, "fp32") == 0


def test_library_has_no_cpu_fallback_symbols(libpath):
    # the product path never reaches the oracle: no oracle symbol in the library
    L = ctypes.CDLL(libpath)
    assert not hasattr(L, "orc_sweep") and not hasattr(L, "orc_create")


C_USER = r"""
#include <stdio.h>
#include "hdmc.h"
int main(void) {
    hdmc_t *h = NULL;
    hdmc3_t *s = NULL;
    double bp = 0.0;
    int e = hdmc_create(&h, 1024, 33.8958, 33.8958, 1.0, 0.15, 4, 1u, HDMC_FP32_LOCAL, NULL, 0, NULL);
    if (e == HDMC_OK) {
        hdmc_sweep(h, 10);
        hdmc_pressure(h, &bp, NULL, NULL, NULL);
        hdmc_destroy(h);
    }
    int e3 = hdmc3_create(&s, 2048, 13.36, 13.36, 13.36, 1.0, 0.1, 4, 1u, HDMC_FP64, NULL, NULL);
    if (e3 == HDMC_OK) hdmc3_destroy(s);
    printf("%d %d %d\n", e, e3, hdmc_build_flags());
    return (e != HDMC_OK && h != NULL) || (e3 != HDMC_OK && s != NULL) ? 3 : 0;   /* *out is NULL on failure */
}
"""


def test_header_is_plain_c_and_links(libpath, tmp_path):
    # a C99 caller (pedantic, warnings as errors) compiles and links against
    # libhdmc.so; the header also compiles as C++.  Run here, where there may
    # be no GPU, it must fail cleanly with an error code (no crash).
    import subprocess
    src = tmp_path / "use.c"
    src.write_text(C_USER)
    exe = tmp_path / "use"
    libdir = os.path.dirname(libpath)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                           os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lhdmc",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-x",
                           "c++", str(src), "-fsyntax-only"])
    import torch
    if torch.cuda.is_available():
        return
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    e, e3, flags = map(int, r.stdout.split())
    assert e != 0 and e3 != 0 and flags == 0


C_GPU_USER = r"""
#include <stdio.h>
#include <inttypes.h>
#include "hdmc.h"
int main(void) {
    hdmc_t *h = NULL;
    double bp = 0.0, g0 = 0.0;
    uint64_t hist[HDMC_HIST_BINS];
    int64_t ns = 0;
    int e = hdmc_create(&h, 1024, 33.89580, 33.89580, 1.0, 0.15, 4, 1u, HDMC_FP32_LOCAL, NULL, 0, NULL);
    if (e != HDMC_OK) { printf("create %d\n", e); return 1; }
    e = hdmc_sweep(h, 10);
    if (e == HDMC_OK) e = hdmc_pressure(h, &bp, &g0, hist, &ns);
    hdmc_destroy(h);
    if (e != HDMC_OK) { printf("error %d\n", e); return 2; }
    printf("%.17g %.17g %" PRId64, bp, g0, ns);
    for (int i = 0; i < HDMC_HIST_BINS; ++i) printf(" %" PRIu64, hist[i]);
    printf("\n");
    return 0;
}
"""


@pytest.mark.gpu
def test_c_caller_on_gpu_matches_oracle(libpath, tmp_path):
    # A plain C99 program drives the library through the C ABI alone (create,
    # 10 binary32 sweeps, pressure): its contact histogram is bit-identical to
    # the oracle's after the same sweeps, and its pressure is the Sec. 4 fit.
    import subprocess
    import oracle as O
    from oracle import pressure as P
    src = tmp_path / "gpu_user.c"
    src.write_text(C_GPU_USER)
    exe = tmp_path / "gpu_user"
    libdir = os.path.dirname(libpath)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                           os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lhdmc",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    f = r.stdout.split()
    bp, ns = float(f[0]), int(f[2])
    hist = np.array([int(x) for x in f[3:]], dtype=np.uint64)
    ref = O.System(1024, 33.89580, 33.89580, 1.0, 0.15, 4, 1, O.FP32)
    ref.sweep(10)
    href = ref.histogram(200, 1e-4)
    assert ns == 1 and hist.sum() > 0 and np.array_equal(hist, href)
    bp_ref = P.pressure(href, 1, 1024, 33.89580 * 33.89580)[0]
    assert abs(bp - bp_ref) < 1e-9 * abs(bp_ref), (bp, bp_ref)

