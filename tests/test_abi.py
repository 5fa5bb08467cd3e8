"""The C ABI (CPU only): libhdmc.so builds, loads, and exports every entry
point include/hdmc.h declares; the Python binding declares the same set.
No compute call is made here (there may be no GPU)."""
import ctypes
import os
import re

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
