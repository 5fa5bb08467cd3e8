"""Snapshots (hdmc_save / hdmc_load): checkpoint and resume through the C ABI.

The random draws are addressed by (seed, sweep, cell, set) counters, so a
restored image must continue bit for bit: positions, slot order, counters,
grid origin and the histogram accumulator, and it must agree with the oracle
run straight through.  Images that break the cell rules are rejected on the
device and leave the handle's state as it was.
"""
import struct

import numpy as np
import pytest

import oracle as O
from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PREC = {"fp64": O.FP64, "fp32": O.FP32}
HEADER = struct.Struct("<8sIIq4d4i4I2Qq5Q")
FIELDS = ("magic version precision N Lx Ly sigma d nsel mx my nblocks key0 key1 flags pad sweeps shifts "
          "n_samples off_state off_partial off_hist off_cells total").split()


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


def _header(buf):
    return dict(zip(FIELDS, HEADER.unpack_from(bytes(buf[:HEADER.size]))))


def _cells(buf, prec):
    """Writable view of the image's cells: (C, 8) = x0..x3, y0..y3."""
    hd = _header(buf)
    dt = np.float64 if prec == "fp64" else np.float32
    C = hd["mx"] * hd["my"]
    return buf[hd["off_cells"]:hd["off_cells"] + C * 8 * np.dtype(dt).itemsize].view(dt).reshape(C, 8)


def _same_run(a, b):
    assert np.array_equal(a.state()[0], b.state()[0])
    assert np.array_equal(a.state()[1], b.state()[1])
    assert np.array_equal(a.counters(), b.counters())
    assert np.array_equal(a.origin(), b.origin())
    assert a.info()["sweeps_done"] == b.info()["sweeps_done"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_snapshot_resume_is_bit_identical_and_matches_oracle(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    a = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 12, prec)
    a.sweep(70)
    a.sample()
    a.sample()
    img = a.save()
    hd = _header(img)
    assert hd["magic"] == b"HDMCSNP1" and hd["N"] == w.N and hd["sweeps"] == 70 and hd["n_samples"] == 2
    assert img.nbytes == a.snapshot_bytes() == hd["total"]

    # a handle of another seed and move size takes both from the image
    b = hdmc.System(w.N, w.Lx, w.Ly, 1.0, 0.1, 4, 99, prec)
    b.sweep(3)
    b.load(img)
    _same_run(a, b)
    assert np.array_equal(b.save(), img)
    for s in (a, b):
        s.sweep(70)
        s.sample()
    _same_run(a, b)
    pa, pb = a.pressure(), b.pressure()
    assert pa[3] == pb[3] == 3
    assert np.array_equal(pa[2], pb[2]) and pa[0] == pb[0]

    # and the resumed run is the oracle's straight run
    o = O.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 12, PREC[prec])
    o.sweep(140)
    assert np.array_equal(b.state()[0], o.state()[0])
    assert np.array_equal(b.counters(), o.counters())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_snapshot_resume_with_crowded_cells(prec):
    # the paper's cell rule (w just below sqrt(2) sigma) fills cells with up
    # to four disks; a run resumed from an image of such a state is still
    # the oracle's straight run
    from paper_1211_1646_gb300 import hdmc
    N = 4096
    L = W.square_box(N, 0.708)
    a = hdmc.System(N, *L, 1.0, 0.16, 4, 21, prec, cells="sqrt2")
    a.sweep(30)
    img = a.save()
    _, cnt = a.state()
    assert (cnt >= 3).sum() > 20 and (cnt == 4).sum() > 0
    b = hdmc.System(N, *L, 1.0, 0.16, 4, 5, prec, cells="sqrt2")
    b.load(img)
    _same_run(a, b)
    b.sweep(30)
    o = O.System(N, *L, 1.0, 0.16, 4, 21, PREC[prec], cells=O.CELLS_SQRT2)
    o.sweep(60)
    assert np.array_equal(b.state()[0], o.state()[0])
    assert np.array_equal(b.state()[1], o.state()[1])
    assert np.array_equal(b.counters(), o.counters())


def test_snapshot_into_pinned_tensor():
    import torch
    from paper_1211_1646_gb300 import hdmc
    w = W.n65536_phi070()
    a = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 5, "fp32")
    a.sweep(20)
    buf = torch.empty(a.snapshot_bytes(), dtype=torch.uint8, pin_memory=True)
    a.save(buf)
    ref = a.save()
    assert np.array_equal(buf.numpy(), ref)
    a.sweep(20)
    after = a.state()
    a.load(buf)
    a.sweep(20)
    assert np.array_equal(a.state()[0], after[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bad_images_are_rejected_and_state_kept(prec):
    from paper_1211_1646_gb300 import hdmc
    w = W.n1024_phi070()
    src = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 3, prec)
    src.sweep(10)
    good = src.save()
    x = _cells(good, prec)
    occ = x[:, :4] != hdmc.HDMC_EMPTY_SLOT
    cnt = occ.sum(1)
    one = int(np.nonzero(cnt == 1)[0][0])
    two = int(np.nonzero(cnt >= 2)[0][0])
    wx = float(np.float32(src.wx)) if prec == "fp32" else src.wx

    def corrupt(kind):
        img = good.copy()
        c = _cells(img, prec)
        if kind == "magic":
            img[0] ^= 0xFF
        elif kind == "x_at_w":
            c[one, 0] = wx
        elif kind == "negative":
            c[one, 4] = -1e-3
        elif kind == "nan":
            c[one, 0] = np.nan
        elif kind == "gap":            # empty slot 0, occupied slot 1: total unchanged
            c[one, 1], c[one, 5] = c[one, 0], c[one, 4]
            c[one, 0] = c[one, 4] = hdmc.HDMC_EMPTY_SLOT
        elif kind == "half_empty":     # x of slot 1 emptied, y kept
            c[two, 1] = hdmc.HDMC_EMPTY_SLOT
        elif kind == "missing_disk":   # a consistent cell, but N - 1 disks
            k = int(cnt[two]) - 1
            c[two, k] = c[two, 4 + k] = hdmc.HDMC_EMPTY_SLOT
        elif kind == "short":
            return img[:-1]
        return img

    kinds = ["magic", "x_at_w", "negative", "nan", "gap", "half_empty", "missing_disk", "short"]
    dst = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 7, prec)
    ref = hdmc.System(w.N, w.Lx, w.Ly, 1.0, w.d, 4, 7, prec)
    dst.sweep(5)
    ref.sweep(5)
    for kind in kinds:
        with pytest.raises(hdmc.HDMCError) as e:
            dst.load(corrupt(kind))
        assert e.value.code == hdmc.HDMC_EINVAL, kind
        _same_run(dst, ref)
    # the handle still runs on, identically to one that saw no bad image
    dst.sweep(9)
    ref.sweep(9)
    _same_run(dst, ref)
    # an image of another system size is refused
    other = hdmc.System(4096, *W.square_box(4096, 0.70), 1.0, 0.1, 4, 1, prec)
    assert other.snapshot_bytes() > dst.snapshot_bytes()
    with pytest.raises(hdmc.HDMCError) as e:
        dst.load(other.save())
    assert e.value.code == hdmc.HDMC_EINVAL
    _same_run(dst, ref)
    dst.load(good)
    _same_run(dst, src)
