"""The contact histogram entry point that allocates nothing.

Callers that cannot allocate device memory (inside another framework's
memory pool, a memory-capped process, a plugin owning no GPU allocations)
use hdmc_histogram_noalloc: it reads a device copy of the state that the
caller owns and keeps its only scratch in a fixed array inside the library.
Its counts must equal those of the library's regular path (hdmc_pressure)
and the oracle's histogram, bit for bit, on two calls in a row.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _widths(g, prec):
    if prec == "fp64":
        return g.wx, g.wy
    return float(np.float32(g.wx)), float(np.float32(g.wy))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_histogram_equals_regular_path_and_oracle(prec):
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    w = W.n65536_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 3, prec)
    ref = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 3, O.FP64 if prec == "fp64" else O.FP32)
    stream = torch.cuda.current_stream().cuda_stream
    wx, wy = _widths(g, prec)
    for call in range(2):
        g.sweep(10)
        ref.sweep(10)
        loc, _ = g.state()
        dev = torch.from_numpy(np.ascontiguousarray(loc.reshape(-1))).to("cuda")
        got = hdmc.hdmc_histogram_noalloc(dev.data_ptr(), g.mx, g.my, wx, wy, 1.0, hdmc.HDMC_HIST_BINS, 1e-4, stream)
        _, _, regular, ns = g.pressure()
        assert ns == 1 and regular.sum() > 0
        assert np.array_equal(got, regular), "call %d" % call
        assert np.array_equal(got, ref.histogram(200, 1e-4)), "call %d" % call


def test_noalloc_largest_size_and_any_negative_empty_slot():
    # nbins = HDMC_NOALLOC_MAX_BINS with dr = 1e-4 reaches sigma + 0.1024,
    # inside two cell widths; its first 200 bins are the regular histogram.
    # Empty slots may hold any negative x: (-0.5, 0.3) gives the same counts.
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    w = W.n65536_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 5, "fp64")
    g.sweep(20)
    loc, cnt = g.state()
    stream = torch.cuda.current_stream().cuda_stream
    nmax = hdmc.HDMC_NOALLOC_MAX_BINS
    dev = torch.from_numpy(np.ascontiguousarray(loc.reshape(-1))).to("cuda")
    full = hdmc.hdmc_histogram_noalloc(dev.data_ptr(), g.mx, g.my, g.wx, g.wy, 1.0, nmax, 1e-4, stream)
    _, _, regular, _ = g.pressure()
    assert full.shape == (nmax,) and np.array_equal(full[:200], regular)
    assert full[200:].sum() > 0
    # the same counts from the oracle after the same 20 sweeps, up to sigma + 0.1024
    ref = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 5, O.FP64)
    ref.sweep(20)
    assert np.array_equal(full, ref.histogram(nmax, 1e-4))
    odd = loc.copy()
    empty = np.arange(4)[None, :] >= cnt[:, None]
    odd[empty, 0] = -0.5
    odd[empty, 1] = 0.3
    dev2 = torch.from_numpy(np.ascontiguousarray(odd.reshape(-1))).to("cuda")
    got = hdmc.hdmc_histogram_noalloc(dev2.data_ptr(), g.mx, g.my, g.wx, g.wy, 1.0, nmax, 1e-4, stream)
    assert np.array_equal(got, full)


def test_noalloc_rejects_bad_arguments_without_launching():
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    buf = torch.full((8 * 64 * 64 + 2,), hdmc.HDMC_EMPTY_SLOT, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    for args in [
        (base, 64, 64, 1.0, 1.0, 1.0, hdmc.HDMC_NOALLOC_MAX_BINS + 1, 1e-4),   # above the maximum size
        (base + 8, 64, 64, 1.0, 1.0, 1.0, 200, 1e-4),                            # 8-byte aligned only
        (base, 64, 64, 1.0, 1.0, 1.0, 1000, 1.0001e-3),                          # sigma + nbins dr > 2 w
        (base, 3, 64, 1.0, 1.0, 1.0, 200, 1e-4),                                 # grid too small
    ]:
        with pytest.raises(hdmc.HDMCError) as e:
            hdmc.hdmc_histogram_noalloc(*args)
        assert e.value.code == hdmc.HDMC_EINVAL, args
    # exactly at the 2 w limit is accepted
    assert hdmc.hdmc_histogram_noalloc(base, 64, 64, 1.0, 1.0, 1.0, 1000, 1e-3).sum() == 0
