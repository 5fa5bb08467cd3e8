"""The contact histogram entry point that allocates nothing.

Callers that cannot allocate device memory (inside another framework's
memory pool, a memory-capped process, a plugin owning no GPU allocations)
use hdmc_histogram_noalloc: it reads a device copy of the state that the
caller owns and keeps its only scratch in a fixed array inside the library.
Its counts must equal those of the library's regular path (hdmc_pressure),
bit for bit, on two calls in a row.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_histogram_equals_regular_path(prec):
    import torch
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    w = W.n65536_phi070()
    g = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, w.nselect, 3, prec)
    stream = torch.cuda.current_stream().cuda_stream
    wx = g.wx if prec == "fp64" else float(np.float32(g.wx))
    wy = g.wy if prec == "fp64" else float(np.float32(g.wy))
    for call in range(2):
        g.sweep(10)
        loc, _ = g.state()
        dev = torch.from_numpy(np.ascontiguousarray(loc.reshape(-1))).to("cuda")
        got = hdmc.hdmc_histogram_noalloc(dev.data_ptr(), g.mx, g.my, wx, wy, 1.0, hdmc.HDMC_HIST_BINS, 1e-4, stream)
        _, _, ref, ns = g.pressure()
        assert ns == 1 and ref.sum() > 0
        assert np.array_equal(got, ref), "call %d" % call


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_1211_1646_gb300 import build, hdmc
    build.build()
    with pytest.raises(hdmc.HDMCError) as e:
        hdmc.hdmc_histogram_noalloc(1, 64, 64, 1.0, 1.0, 1.0, hdmc.HDMC_NOALLOC_MAX_BINS + 1, 1e-4)
    assert e.value.code == hdmc.HDMC_EINVAL
