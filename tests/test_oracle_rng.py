"""Pins for the oracle's random streams (CPU only).

Philox4x32-10 is checked against an independent implementation (triton's
philox, run in triton's CPU interpreter), and the derived draws against the
distributions they must have: exact uniformity of the bounded integers over
every 32-bit word, exact mirror symmetry of the displacement lattice,
uniformity in the unit disk, uniform permutations, and the sweep-level draws
of Alg. 1.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle as O

from golden import keyvals

_TRITON_SCRIPT = r"""
import json, sys
import torch, triton, triton.language as tl
cases = json.loads(sys.stdin.read())
@triton.jit
def k(out, seed, c0p, c1p, c2p, c3p, n: tl.constexpr):
    o = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o), tl.load(c2p + o), tl.load(c3p + o))
    tl.store(out + 4 * o + 0, a)
    tl.store(out + 4 * o + 1, b)
    tl.store(out + 4 * o + 2, c)
    tl.store(out + 4 * o + 3, d)
res = []
for seed, ctrs in cases:
    n = len(ctrs)
    cols = [torch.tensor([c[i] for c in ctrs], dtype=torch.uint32) for i in range(4)]
    out = torch.zeros(4 * n, dtype=torch.uint32)
    k[(1,)](out, seed, *cols, n=n)
    res.append([int(x) for x in out])
print(json.dumps(res))
"""


def test_philox_matches_independent_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    cases = []
    for seed in [0, 1, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3, int(rng.integers(0, 2**63))]:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
        ctrs += [[int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)] for _ in range(5)]
        cases.append([seed, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases), env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctrs), out in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i, ctr in enumerate(ctrs):
            mine = O.philox(ctr, key)
            assert [int(x) for x in mine] == out[4 * i: 4 * i + 4], (seed, ctr)


def test_philox_stream_statistics():
    # 2^20 words from 4096 independent streams
    words = np.concatenate([O.stream_words(12345, s, 7, 1 << 28, 256) for s in range(4096)])
    u = words.astype(np.float64) / 2.0**32
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-6
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / math.sqrt(n))
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(n)


def test_philox_avalanche():
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(2000):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        b = int(rng.integers(0, 128))
        ctr2 = ctr.copy()
        ctr2[b // 32] ^= np.uint32(1 << (b % 32))
        x = O.philox(ctr, key) ^ O.philox(ctr2, key)
        flips.append(sum(bin(int(v)).count("1") for v in x))
    assert abs(np.mean(flips) - 64) < 1.0


@pytest.mark.parametrize("rng_range", [3, 4])
def test_bounded_integers_exactly_uniform(rng_range):
    # every 32-bit word, through the same mapping the streams use
    counts = O.lemire_exhaustive(rng_range)
    assert len(set(int(c) for c in counts)) == 1
    assert int(counts[0]) == (2**32) // rng_range


@pytest.mark.parametrize("rng_range", [2, 3, 5, 24])
def test_bounded_stream_uniform(rng_range):
    v = O.stream_bounded(99, 1, 2, 3, rng_range, 240000)
    assert v.max() < rng_range
    counts = np.bincount(v.astype(np.int64), minlength=rng_range)
    assert stats.chisquare(counts).pvalue > 1e-6


def test_symmetric_variates_exact_mirror():
    L = O.lib()
    rng = np.random.default_rng(11)
    for _ in range(20000):
        hi, lo = (int(x) for x in rng.integers(0, 2**32, 2, dtype=np.uint64))
        u = L.orc_sym52(hi, lo)
        assert L.orc_sym52(hi ^ 0xFFFFFFFF, lo ^ 0xFFFFFFFF) == -u
        assert -1.0 < u < 1.0
        m = u * 2.0**52
        assert m == math.floor(m) and int(m) % 2 == 1
    # extremes of the lattice
    assert L.orc_sym52(0, 0) == -(1 - 2.0**-52)
    assert L.orc_sym52(0xFFFFFFFF, 0xFFFFFFFF) == 1 - 2.0**-52


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_displacement_uniform_in_unit_disk(prec):
    uv = np.concatenate([O.displacements(5, s, 1, 2, prec, 50000) for s in range(4)])
    r2 = (uv**2).sum(axis=1)
    assert np.all(r2 < 1.0)
    # uniform in the disk <=> r^2 ~ U(0,1) and angle ~ U(0, 2 pi), independent
    assert stats.kstest(r2, "uniform").pvalue > 1e-4
    th = (np.arctan2(uv[:, 1], uv[:, 0]) + np.pi) / (2 * np.pi)
    assert stats.kstest(th, "uniform").pvalue > 1e-4
    rings = np.minimum((r2 * 8).astype(int), 7)
    sectors = np.minimum((th * 8).astype(int), 7)
    tab = np.bincount(rings * 8 + sectors, minlength=64)
    assert stats.chisquare(tab).pvalue > 1e-6
    assert abs(uv[:, 0].mean()) < 5 * 0.5 / math.sqrt(len(uv))


@pytest.mark.parametrize("rng_range", [2, 6, 24])
def test_bounded_21bit_fields_exactly_uniform(rng_range):
    counts = O.lemire21_exhaustive(rng_range)
    assert len(set(int(c) for c in counts)) == 1
    assert int(counts[0]) == (2**21) // rng_range


def test_21bit_fields_and_variates():
    L = O.lib()
    rng = np.random.default_rng(12)
    for _ in range(2000):
        w = rng.integers(0, 2**32, 4, dtype=np.uint64)
        big = int(w[0]) | int(w[1]) << 32 | int(w[2]) << 64 | int(w[3]) << 96
        f = O.fields21(w)
        assert [int(x) for x in f] == [(big >> (21 * j)) & 0x1FFFFF for j in range(6)]
    for k in range(0, 2**21, 997):
        u = L.orc_sym21(k)
        assert L.orc_sym21(k ^ 0x1FFFFF) == -u and -1 < u < 1
        assert (u * 2**21) % 2 == 1
    assert L.orc_sym21(0) == -(1 - 2.0**-21)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_permutation_decode_is_a_bijection(n):
    seen = {tuple(int(x) for x in O.decode_perm(n, k)) for k in range(math.factorial(n))}
    assert len(seen) == math.factorial(n)
    assert all(sorted(p) == list(range(n)) for p in seen)


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
@pytest.mark.parametrize("n", [2, 3, 4])
def test_fisher_yates_uniform_permutations(n, prec):
    perms = O.shuffles(17, 3, 2, n, 120000, prec)
    assert np.all(np.sort(perms, axis=1) == np.arange(n))
    code = np.zeros(len(perms), dtype=np.int64)
    for j in range(n):
        code = code * n + perms[:, j]
    _, counts = np.unique(code, return_counts=True)
    assert len(counts) == math.factorial(n)
    assert stats.chisquare(counts).pvalue > 1e-6


def test_sweep_level_draws():
    wx, wy = 1.0592437756635953, 1.0004
    perms, fs, ds = [], [], []
    for s in range(24000):
        p, f, d = O.sweep_draws(1, s, wx, wy)
        perms.append(tuple(int(v) for v in p))
        fs.append(f)
        ds.append(d / (0.5 * (wy if f >= 2 else wx)))
    assert all(sorted(p) == [0, 1, 2, 3] for p in perms)
    _, pc = np.unique(np.array(perms), axis=0, return_counts=True)
    assert len(pc) == 24 and stats.chisquare(pc).pvalue > 1e-6
    assert stats.chisquare(np.bincount(fs, minlength=4)).pvalue > 1e-6
    ds = np.array(ds)
    assert ds.min() >= 0.0 and ds.max() < 1.0
    assert stats.kstest(ds, "uniform").pvalue > 1e-4


def test_visit_order_matches_paper_example():
    g = keyvals("reverse_sequence_sec2_3.txt")
    n, nM = g["n"], g["n_M"]
    fwd = O.visit_sequence(n, nM)
    assert list(fwd) == g["forward"]
    # among all shufflings, exactly one reverses the sequence (Sec. 2.3)
    import itertools
    hits = []
    for perm in itertools.permutations(range(n)):
        seq = [perm[i] for i in fwd]
        if seq == list(reversed([int(x) for x in fwd])):
            hits.append(list(perm))
    assert hits == [g["reverse_shuffle"]]
    assert [g["reverse_shuffle"][i] for i in fwd] == g["reverse"]
