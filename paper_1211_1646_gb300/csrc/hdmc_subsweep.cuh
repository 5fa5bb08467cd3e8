// hdmc_subsweep.cuh -- the sub-sweep kernels (Alg. 2) in binary32 and
// binary64.
//
// Every floating-point operation that decides an acceptance is written with
// an explicit round-to-nearest operation, so the result does not depend on
// compiler contraction:
//   binary64: trial coordinate p + d*u, overlap iff dx*dx + dy*dy < sigma^2;
//   binary32: trial coordinate fma(d, u, p), overlap iff
//             fma(dx, dx, fma(dy, dy, -sigma^2)) < 0.
#pragma once

#include "hdmc_common.cuh"

namespace hdmc {

// ---- binary32 sub-sweep: the cell updates of Alg. 1 / Alg. 2 ---------------------------
// One thread per active cell of set Q = draw->perm[k]; block 32 x ROWS over
// the set's half-resolution grid.  Phases, ordered so that the latency of the
// cell loads is covered by work that does not need them:
//   1. issue the loads of the own cell and of the 8 neighbouring cells (they
//      belong to other sets and are not written by this launch);
//   2. draw the trial directions of the cell's stream (kept attempts staged
//      in shared memory, kDirChunk at a time);
//   3. shuffle the disks with the draw in field 0 of the stream's first block,
//      translate neighbour slot pair (0,1) into this cell's frame as packed
//      binary32 pairs, flag (warp-uniformly) the directions where some lane
//      has a third disk;
//   4. n_M trial moves, visiting the shuffled slots cyclically.
// NSEL > 0 fixes n_M at compile time (the trial loop is then unrolled).
// With TRACK, the block also adds the net squared displacement of its disks
// over the cell update (final minus start position, summed over the disks)
// to *msd: a sampling-efficiency measure used by the batch autotuner.
template <int ROWS>
__device__ __forceinline__ void draw_directions(const Geometry& g, uint32_t sweep, uint32_t cell, uint32_t c2,
                                                uint32_t F[6], uint32_t& blk, int& pnext, int want,
                                                float2 (*__restrict__ sdir)[32 * ROWS], int tid) {
    int have = 0;
    for (;;) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (p >= pnext && have < want) {
                const float u = sym21(F[2 * p]), v = sym21(F[2 * p + 1]);
                if (__fmaf_rn(u, u, __fmul_rn(v, v)) < 1.0f) {
                    sdir[have][tid] = make_float2(u, v);
                    ++have;
                }
                pnext = p + 1;
            }
        }
        if (have >= want) break;
        ++blk;
        fields21(philox4x32_10(make_uint4(sweep, cell, c2, blk), g.key0, g.key1), F);
        pnext = 0;
    }
}

// Philox4x32-10 (the library's philox4x32_10, the same function) with the
// round keys of one key computed once per thread.  WIDE forms each round's
// two products as 32 x 32 -> 64-bit multiplies, otherwise as separate high
// and low products (measured: the wide form is faster in the n_M = 8
// kernels, the separate one in the n_M = 4 kernels).
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
    __device__ __forceinline__ PhiloxKeys(uint32_t a, uint32_t b) {
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            k0[r] = a + (uint32_t)r * 0x9E3779B9u;
            k1[r] = b + (uint32_t)r * 0xBB67AE85u;
        }
    }
};
template <bool WIDE>
__device__ __forceinline__ uint4 philox_rk(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        if constexpr (WIDE) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
            hi0 = (uint32_t)(p0 >> 32);
            lo0 = (uint32_t)p0;
            hi1 = (uint32_t)(p1 >> 32);
            lo1 = (uint32_t)p1;
        } else {
            hi0 = __umulhi(0xD2511F53u, c.x);
            lo0 = 0xD2511F53u * c.x;
            hi1 = __umulhi(0xCD9E8D57u, c.z);
            lo1 = 0xCD9E8D57u * c.z;
        }
        c = make_uint4(hi1 ^ c.y ^ K.k0[r], lo1, hi0 ^ c.w ^ K.k1[r], lo0);
    }
    return c;
}

// All WANT <= kDirChunk directions of a cell update in one pass, in the
// stream order of draw_directions: the two attempts of block 0 (field pairs
// 1 and 2), blocks 1 and 2 without a loop (every lane needs block 1 and
// nearly every warp has a lane that needs block 2), then block after block
// while the lane has fewer than WANT kept attempts.  A lane may keep more
// than WANT (at most max(8, WANT + 2) <= kDirRows), in rows of sdir that no
// trial reads; the stream is not continued.
template <int ROWS, int WANT>
__device__ __forceinline__ void draw_directions_once(const PhiloxKeys& K, uint32_t sweep, uint32_t cell, uint32_t c2,
                                                     const uint32_t F0[6], float2 (*__restrict__ sdir)[32 * ROWS],
                                                     int tid) {
    static_assert(WANT <= kDirChunk && kDirRows >= kDirChunk + 2 && kDirRows >= 8, "sdir rows");
    int have = 0;
    auto attempt = [&](uint32_t a, uint32_t b) {
        const float u = sym21(a), v = sym21(b);
        if (__fmaf_rn(u, u, __fmul_rn(v, v)) < 1.0f) {
            sdir[have][tid] = make_float2(u, v);
            ++have;
        }
    };
    attempt(F0[2], F0[3]);
    attempt(F0[4], F0[5]);
#pragma unroll
    for (uint32_t blk = 1; blk < 3; ++blk) {   // every lane needs block 1, nearly every warp block 2
        uint32_t F[6];
        fields21(philox_rk<(WANT > 4)>(make_uint4(sweep, cell, c2, blk), K), F);
        attempt(F[0], F[1]);
        attempt(F[2], F[3]);
        attempt(F[4], F[5]);
    }
    for (uint32_t blk = 3; have < WANT; ++blk) {
        uint32_t F[6];
        fields21(philox_rk<(WANT > 4)>(make_uint4(sweep, cell, c2, blk), K), F);
        attempt(F[0], F[1]);
        attempt(F[2], F[3]);
        attempt(F[4], F[5]);
    }
}

// DENSE (cells that often hold three or four disks, as with the paper's
// cells just below sqrt(2) sigma): slot pairs (2,3) of all 8 neighbours stay
// in registers and every trial tests all of them, instead of the flagged
// directions' pairs being read again in every trial.
template <int ROWS, int NSEL, bool TRACK = false, bool DENSE = false>
__device__ __forceinline__ void subsweep_f32(const Geometry& g, float* __restrict__ cells,
                                             const SweepDraw* __restrict__ draw, int k, int bx, int by,
                                             unsigned long long* __restrict__ bpart,
                                             float2 (*__restrict__ sdir)[32 * ROWS], double* msd = nullptr) {
    const int nsel = NSEL > 0 ? NSEL : g.nsel;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int Q = draw->perm[k];
    const uint32_t sweep = draw->sweep;
    const int hx = bx * 32 + threadIdx.x;
    const int hy = by * ROWS + threadIdx.y;
    const int cx = 2 * hx + (Q & 1), cy = 2 * hy + (Q >> 1);
    const bool live = hx < g.hx && hy < g.hy && cy >= g.ylo && cy <= g.yhi;
    const Neighbourhood nbh(g, Q, hx, hy, live);

    // 1. loads
    Cell<float> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = (float)kEmpty;
    float* ownp = cell_at(cells, nbh.own(g, hx, hy));
    if (live) load_cell(ownp, own);
    float4 n01[8];   // slots 0,1 of the neighbours (x0 x1 y0 y1); slot 2 only to flag its use
    float n2[8];
    float4 n23[DENSE ? 8 : 1];   // DENSE: slots 2,3 of the neighbours (x2 x3 y2 y3)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        n01[c] = make_float4((float)kEmpty, (float)kEmpty, (float)kEmpty, (float)kEmpty);
        n2[c] = (float)kEmpty;
        if (DENSE) n23[c] = n01[c];
        if (live) {
            const float* p = cell_at(cells, nbh.index(g, c, hx, hy));
            Cell<float> a;
            load_cell_ro(p, a);   // one 256-bit load; slots 0, 1 and x2 are used
            n01[c] = make_float4(a.x[0], a.x[1], a.y[0], a.y[1]);
            n2[c] = a.x[2];
            if (DENSE) n23[c] = make_float4(a.x[2], a.x[3], a.y[2], a.y[3]);
        }
    }

    // 2. directions of the first chunk (the cell's trial stream)
    const uint32_t cell = (uint32_t)(cy + g.row0) * (uint32_t)g.mx + (uint32_t)cx;   // global cell number
    const uint32_t c2 = (kDomTrial << 28) | ((uint32_t)Q << 24);
    uint32_t F[6];
    uint32_t f0;                 // shuffle draw: field 0 of block 0
    uint32_t blk = 0;
    int pnext = 1;               // next attempt: field pair 1 of block 0 (fields 2,3)
    if constexpr (NSEL > 0 && NSEL <= kDirChunk) {
        const PhiloxKeys K(g.key0, g.key1);
        fields21(philox_rk<(NSEL > 4)>(make_uint4(sweep, cell, c2, 0u), K), F);
        f0 = F[0];
        draw_directions_once<ROWS, NSEL>(K, sweep, cell, c2, F, sdir, tid);
    } else {
        fields21(philox4x32_10(make_uint4(sweep, cell, c2, 0u), g.key0, g.key1), F);
        f0 = F[0];
        draw_directions<ROWS>(g, sweep, cell, c2, F, blk, pnext, min(kDirChunk, nsel), sdir, tid);   // refills F
    }

    // 3. cell contents
    const int n = (own.x[0] >= 0.f) + (own.x[1] >= 0.f) + (own.x[2] >= 0.f) + (own.x[3] >= 0.f);
    uint32_t dir23 = 0;   // warp-uniform: directions where some lane has a third disk
    {
        uint32_t mine = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) mine |= (n2[c] >= 0.f) ? (1u << c) : 0u;
        dir23 = __reduce_or_sync(0xffffffffu, mine);
    }
    const bool own23 = __any_sync(0xffffffffu, n >= 3);

    unsigned int n_tr = 0, n_acc = 0, n_leave = 0;
    float net2 = 0.f;
    if (n > 0) {
        // shuffle of the cell's disks (Alg. 1): one draw in [0, n!) by 21-bit Lemire on field 0
        if (n >= 2 && !(g.flags & kNoParticleShuffle)) {
            const uint32_t range = factorial(n);
            const uint32_t m = f0 * range;
            const uint32_t thr = n == 4 ? 8u : (n == 3 ? 2u : 0u);   // 2^21 mod n!
            uint32_t kk = m >> 21;
            if ((m & 0x1FFFFFu) < thr) {   // rejected: draw from the shuffle stream instead
                WordStream s(g.key0, g.key1, sweep, cell, (kDomShuffle << 28) | ((uint32_t)Q << 24));
                kk = s.bounded(range);
            }
            shuffle_slots(own.x, own.y, n, kk);
        }
        float sx0[4], sy0[4];
        if (TRACK) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                sx0[j] = own.x[j];
                sy0[j] = own.y[j];
            }
        }
        f2x qx01[8], qy01[8];
        f2x qx23[DENSE ? 8 : 1], qy23[DENSE ? 8 : 1];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float sx = (float)dir_dx(c) * g.wxf, sy = (float)dir_dy(c) * g.wyf;
            qx01[c] = add2(pk(n01[c].x, n01[c].y), pk(sx, sx));
            qy01[c] = add2(pk(n01[c].z, n01[c].w), pk(sy, sy));
            if (DENSE) {
                qx23[c] = add2(pk(n23[c].x, n23[c].y), pk(sx, sx));
                qy23[c] = add2(pk(n23[c].z, n23[c].w), pk(sy, sy));
            }
        }
        // slot pair (2,3) of the first flagged direction, translated; further
        // flagged directions (rare) are read in the trial loop
        f2x fx23 = 0, fy23 = 0;
        const uint32_t more23 = DENSE ? 0u : dir23 & (dir23 - 1);
        if (!DENSE && dir23) {
            const int c = __ffs(dir23) - 1;
            const float2* p = reinterpret_cast<const float2*>(cell_at(cells, nbh.index(g, c, hx, hy)));
            const float2 x23 = __ldg(p + 1), y23 = __ldg(p + 3);
            const float sx = (float)dir_dx(c) * g.wxf, sy = (float)dir_dy(c) * g.wyf;
            fx23 = add2(pk(x23.x, x23.y), pk(sx, sx));
            fy23 = add2(pk(y23.x, y23.y), pk(sy, sy));
        }
        const float df = g.df;
        const f2x ns2 = pk(-g.sig2f, -g.sig2f);

        // 4. trials; trial tt of the current chunk uses direction sdir[tt]
        // and slot i, which lies in the slot set M
        int i = 0;
        auto trial = [&](int tt, auto slots) {
            constexpr unsigned M = decltype(slots)::value;
            {
                const float2 uv = sdir[tt][tid];
                const float tx = __fmaf_rn(df, uv.x, pick_in<M>(own.x, i));
                const float ty = __fmaf_rn(df, uv.y, pick_in<M>(own.y, i));
                // tx >= 0 && tx < w as one unsigned compare of the bit
                // patterns (w > 0); exact because fma(d, u, p) with
                // d*u != 0 is never -0, the one value read differently
                const bool inside = __float_as_uint(tx) < __float_as_uint(g.wxf) &&
                                    __float_as_uint(ty) < __float_as_uint(g.wyf);
                const f2x tx2 = pk(tx, tx), ty2 = pk(ty, ty);
                // own cell: every other occupied slot (slot i excluded)
                f2x z = zpair(tx2, ty2, pk(own.x[0], own.x[1]), pk(own.y[0], own.y[1]), ns2);
                uint32_t acc = ((M & 1u) && i == 0 ? 0u : lo32(z)) | ((M & 2u) && i == 1 ? 0u : hi32(z));
                if (DENSE || own23) {
                    z = zpair(tx2, ty2, pk(own.x[2], own.x[3]), pk(own.y[2], own.y[3]), ns2);
                    acc |= ((M & 4u) && i == 2 ? 0u : lo32(z)) | ((M & 8u) && i == 3 ? 0u : hi32(z));
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    z = zpair(tx2, ty2, qx01[c], qy01[c], ns2);
                    acc |= lo32(z) | hi32(z);
                    if (DENSE) {
                        z = zpair(tx2, ty2, qx23[c], qy23[c], ns2);
                        acc |= lo32(z) | hi32(z);
                    }
                }
                if (!DENSE && dir23) {
                    z = zpair(tx2, ty2, fx23, fy23, ns2);
                    acc |= lo32(z) | hi32(z);
                }
                for (uint32_t m = more23; m; m &= m - 1) {   // warp-uniform, rarely taken
                    const int c = __ffs(m) - 1;
                    const float2* p = reinterpret_cast<const float2*>(cell_at(cells, nbh.index(g, c, hx, hy)));
                    const float2 x23 = __ldg(p + 1), y23 = __ldg(p + 3);
                    const float sx = (float)dir_dx(c) * g.wxf, sy = (float)dir_dy(c) * g.wyf;
                    z = zpair(tx2, ty2, add2(pk(x23.x, x23.y), pk(sx, sx)), add2(pk(y23.x, y23.y), pk(sy, sy)), ns2);
                    acc |= lo32(z) | hi32(z);
                }
                const bool ok = inside && !(acc & 0x80000000u);
                put_in<M>(own.x, i, tx, ok);
                put_in<M>(own.y, i, ty, ok);
                n_acc += ok;
                n_leave += !inside;
                i = (i + 1 == n) ? 0 : i + 1;
            }
        };
        if constexpr (NSEL > 0 && NSEL <= kDirChunk) {
            unrolled_trials(trial, std::make_integer_sequence<int, NSEL>{});
        } else {
            for (int t0 = 0; t0 < nsel; t0 += kDirChunk) {
                const int want = min(kDirChunk, nsel - t0);
                if (t0 > 0) draw_directions<ROWS>(g, sweep, cell, c2, F, blk, pnext, want, sdir, tid);
#pragma unroll 1
                for (int tt = 0; tt < want; ++tt) trial(tt, std::integral_constant<unsigned, 0xFu>{});
            }
        }
        n_tr = (unsigned)nsel;
        store_cell(ownp, own);
        if (TRACK) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float ex = own.x[j] - sx0[j], ey = own.y[j] - sy0[j];
                net2 += ex * ex + ey * ey;
            }
        }
    }
    if (TRACK) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) net2 += __shfl_xor_sync(0xffffffffu, net2, o);
        if (threadIdx.x == 0) atomicAdd(msd, (double)net2);
    }
    add_block_counters<ROWS>(n_tr, n_acc, n_leave, bpart);
}

template <int ROWS, int NSEL, bool DENSE = false>
static __global__ void __launch_bounds__(32 * ROWS, DENSE ? 16 / ROWS : 20 / ROWS)
k_subsweep_f32(const Geometry g, float* __restrict__ cells, const SweepDraw* __restrict__ draw, int k,
               unsigned long long* __restrict__ partial) {
    pdl_release();
    pdl_wait();
    __shared__ float2 sdir[kDirRows][32 * ROWS];
    // counters of the tile that holds this block (shared by the blocks of a
    // tile: atomic adds)
    const long long slot = (long long)(blockIdx.y * ROWS / kCounterRows) * gridDim.x + blockIdx.x;
    subsweep_f32<ROWS, NSEL, false, DENSE>(g, cells, draw, k, blockIdx.x, blockIdx.y, partial + 4 * slot, sdir);
}

// ---- binary64 sub-sweep ---------------------------------------------------------------
// Same algorithm in binary64.  Draws: shuffle by one 32-bit Lemire draw in
// [0, n!) from the cell's shuffle stream; trial t takes the t-th kept attempt
// of the trial stream, attempt a = block a: u = sym52(w0,w1), v = sym52(w2,w3),
// kept iff u*u + v*v < 1.
//
// Every decision is the exact binary64 expression, but binary64 arithmetic
// is slow on this GPU, so binary32 estimates settle the clear cases first:
//  - in-circle test: u, v truncated to 23 bits (|error| <= 2^-23); cases with
//    the estimate of u^2 + v^2 within 2^-18 of 1 are decided in binary64;
//  - overlap test: positions truncated to binary32 (relative error <= 2^-23),
//    the squared distance estimated with binary32 pair arithmetic (error
//    below 3e-6 where it matters, r^2 < 1.3); a candidate counts as certainly
//    overlapping below sigma^2 - 2^-15 and certainly clear above sigma^2 + 2^-15;
//    if any candidate falls in between, all candidates are tested in binary64.
constexpr float kOverlapBand = 0x1p-15f;
constexpr float kCircleBand = 0x1p-18f;

// Exact binary64 overlap test of a trial position against every candidate
// whose binary32 estimate (the prefilter's own expression, with the upper
// band edge) says "possibly overlapping"; the others are certainly clear.
// sigma^2 and r^2 are non-negative, so r^2 < sigma^2 compares bit patterns.
__device__ __forceinline__ bool exact_trial_hit(const Geometry& g, const double* __restrict__ cells,
                                                  const Neighbourhood& nbh, int hx, int hy, const Cell<double>& own,
                                                  const float ofx[4], const float ofy[4], int i, double tx, double ty,
                                                  float txf, float tyf) {
    const long long s2 = __double_as_longlong(g.sig2);
    const float nhi = -((float)g.sig2 + kOverlapBand);
    bool hit = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float ex = __fsub_rn(txf, ofx[j]), ey = __fsub_rn(tyf, ofy[j]);
        if (j != i && __fmaf_rn(ex, ex, __fmaf_rn(ey, ey, nhi)) < 0.f) {
            const double ddx = __dsub_rn(tx, own.x[j]), ddy = __dsub_rn(ty, own.y[j]);
            hit |= __double_as_longlong(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy))) < s2;
        }
    }
    const float wxf = (float)g.wx, wyf = (float)g.wy;
    for (int c = 0; c < 8; ++c) {
        Cell<double> a;
        load_cell_ro(cell_at(cells, nbh.index(g, c, hx, hy)), a);
        const double sx = (double)dir_dx(c) * g.wx, sy = (double)dir_dy(c) * g.wy;
        const float sxf = (float)dir_dx(c) * wxf, syf = (float)dir_dy(c) * wyf;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float ex = __fsub_rn(txf, __fadd_rn(approx_f32(a.x[j]), sxf));
            const float ey = __fsub_rn(tyf, __fadd_rn(approx_f32(a.y[j]), syf));
            if (__fmaf_rn(ex, ex, __fmaf_rn(ey, ey, nhi)) < 0.f) {
                const double ddx = __dsub_rn(tx, __dadd_rn(a.x[j], sx)), ddy = __dsub_rn(ty, __dadd_rn(a.y[j], sy));
                hit |= __double_as_longlong(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy))) < s2;
            }
        }
    }
    return hit;
}

// 53-bit odd integer m of sym52 (u = m 2^-52) and its binary32 truncation m 2^-52.
__device__ __forceinline__ long long sym52_int(uint32_t hi, uint32_t lo) {
    const unsigned long long k = (((unsigned long long)hi << 32) | lo) >> 12;
    return (long long)(2 * k + 1) - (1ll << 52);
}
__device__ __forceinline__ float sym52_est(long long m) { return (float)(int)(m >> 29) * 0x1p-23f; }

template <int ROWS>
__device__ __forceinline__ void subsweep_f64(const Geometry& g, double* __restrict__ cells,
                                             const SweepDraw* __restrict__ draw, int k, int bx, int by,
                                             unsigned long long* __restrict__ bpart) {
    const int Q = draw->perm[k];
    const uint32_t sweep = draw->sweep;
    const int hx = bx * 32 + threadIdx.x;
    const int hy = by * ROWS + threadIdx.y;
    const int cx = 2 * hx + (Q & 1), cy = 2 * hy + (Q >> 1);
    const bool live = hx < g.hx && hy < g.hy && cy >= g.ylo && cy <= g.yhi;
    const Neighbourhood nbh(g, Q, hx, hy, live);

    Cell<double> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = kEmpty;
    double* ownp = cell_at(cells, nbh.own(g, hx, hy));
    if (live) load_cell(ownp, own);
    float4 n01[8];   // binary32 truncations of neighbour slots 0,1 (x0 x1 y0 y1)
    float n2[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        n01[c] = make_float4((float)kEmpty, (float)kEmpty, (float)kEmpty, (float)kEmpty);
        n2[c] = (float)kEmpty;
        if (live) {
            const double* p = cell_at(cells, nbh.index(g, c, hx, hy));
            const double2 x01 = __ldg(reinterpret_cast<const double2*>(p));
            const double2 y01 = __ldg(reinterpret_cast<const double2*>(p) + 2);
            n01[c] = make_float4(approx_f32(x01.x), approx_f32(x01.y), approx_f32(y01.x), approx_f32(y01.y));
            n2[c] = approx_f32(__ldg(p + 2));
        }
    }
    const int n = Prm<double>::ge0(own.x[0]) + Prm<double>::ge0(own.x[1]) + Prm<double>::ge0(own.x[2]) +
                  Prm<double>::ge0(own.x[3]);
    uint32_t dir23 = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) dir23 |= __any_sync(0xffffffffu, n2[c] >= 0.f) ? (1u << c) : 0u;
    const bool own23 = __any_sync(0xffffffffu, n >= 3);

    unsigned int n_tr = 0, n_acc = 0, n_leave = 0;
    if (n > 0) {
        const uint32_t cell = (uint32_t)(cy + g.row0) * (uint32_t)g.mx + (uint32_t)cx;   // global cell number
        const uint32_t setbits = (uint32_t)Q << 24;
        if (n >= 2 && !(g.flags & kNoParticleShuffle)) {
            WordStream s(g.key0, g.key1, sweep, cell, (kDomShuffle << 28) | setbits);
            shuffle_slots(own.x, own.y, n, s.bounded(factorial(n)));
        }
        float ofx[4], ofy[4];   // binary32 truncations of the own slots
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ofx[j] = approx_f32(own.x[j]);
            ofy[j] = approx_f32(own.y[j]);
        }
        const float wxf = (float)g.wx, wyf = (float)g.wy;
        f2x qx01[8], qy01[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float sx = (float)dir_dx(c) * wxf, sy = (float)dir_dy(c) * wyf;
            qx01[c] = add2(pk(n01[c].x, n01[c].y), pk(sx, sx));
            qy01[c] = add2(pk(n01[c].z, n01[c].w), pk(sy, sy));
        }
        f2x fx23 = 0, fy23 = 0;
        const uint32_t more23 = dir23 & (dir23 - 1);
        if (dir23) {
            const int c = __ffs(dir23) - 1;
            const double2* p = reinterpret_cast<const double2*>(cell_at(cells, nbh.index(g, c, hx, hy)));
            const double2 x23 = __ldg(p + 1), y23 = __ldg(p + 3);
            const float sx = (float)dir_dx(c) * wxf, sy = (float)dir_dy(c) * wyf;
            fx23 = add2(pk(approx_f32(x23.x), approx_f32(x23.y)), pk(sx, sx));
            fy23 = add2(pk(approx_f32(y23.x), approx_f32(y23.y)), pk(sy, sy));
        }
        const float s2f = (float)g.sig2;
        const f2x nlo = pk(-(s2f - kOverlapBand), -(s2f - kOverlapBand));   // certainly overlapping below
        const f2x nhi = pk(-(s2f + kOverlapBand), -(s2f + kOverlapBand));   // possibly overlapping below
        const double dscaled = g.d * 0x1p-52;   // d*u = (d 2^-52) * m exactly as real numbers
        const uint32_t c2 = (kDomTrial << 28) | setbits;
        uint32_t blk = 0;
        int i = 0;
        for (int t = 0; t < g.nsel; ++t) {
            long long mu, mv;
            for (;;) {
                const uint4 r = philox4x32_10(make_uint4(sweep, cell, c2, blk++), g.key0, g.key1);
                mu = sym52_int(r.x, r.y);
                mv = sym52_int(r.z, r.w);
                const float uf = sym52_est(mu), vf = sym52_est(mv);
                const float e = __fmaf_rn(uf, uf, __fmul_rn(vf, vf));
                if (e < 1.0f - kCircleBand) break;
                if (e >= 1.0f + kCircleBand) continue;
                const double u = (double)mu * 0x1p-52, v = (double)mv * 0x1p-52;
                if (__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)) < 1.0) break;
            }
            const double tx = __dadd_rn(pick(own.x, i), __dmul_rn(dscaled, (double)mu));
            const double ty = __dadd_rn(pick(own.y, i), __dmul_rn(dscaled, (double)mv));
            const bool inside = Prm<double>::ge0(tx) && Prm<double>::lt(tx, g.wx) && Prm<double>::ge0(ty) &&
                                Prm<double>::lt(ty, g.wy);
            const float txf = approx_f32(tx), tyf = approx_f32(ty);
            const f2x tx2 = pk(txf, txf), ty2 = pk(tyf, tyf);
            uint32_t sure = 0, maybe = 0;   // sign bits: certainly / possibly overlapping
            {
                const f2x dx = sub2(tx2, pk(ofx[0], ofx[1])), dy = sub2(ty2, pk(ofy[0], ofy[1]));
                const f2x zl = fma2(dx, dx, fma2(dy, dy, nlo)), zh = fma2(dx, dx, fma2(dy, dy, nhi));
                sure |= (i == 0 ? 0u : lo32(zl)) | (i == 1 ? 0u : hi32(zl));
                maybe |= (i == 0 ? 0u : lo32(zh)) | (i == 1 ? 0u : hi32(zh));
            }
            if (own23) {
                const f2x dx = sub2(tx2, pk(ofx[2], ofx[3])), dy = sub2(ty2, pk(ofy[2], ofy[3]));
                const f2x zl = fma2(dx, dx, fma2(dy, dy, nlo)), zh = fma2(dx, dx, fma2(dy, dy, nhi));
                sure |= (i == 2 ? 0u : lo32(zl)) | (i == 3 ? 0u : hi32(zl));
                maybe |= (i == 2 ? 0u : lo32(zh)) | (i == 3 ? 0u : hi32(zh));
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const f2x dx = sub2(tx2, qx01[c]), dy = sub2(ty2, qy01[c]);
                const f2x zl = fma2(dx, dx, fma2(dy, dy, nlo)), zh = fma2(dx, dx, fma2(dy, dy, nhi));
                sure |= lo32(zl) | hi32(zl);
                maybe |= lo32(zh) | hi32(zh);
            }
            if (dir23) {
                const f2x dx = sub2(tx2, fx23), dy = sub2(ty2, fy23);
                const f2x zl = fma2(dx, dx, fma2(dy, dy, nlo)), zh = fma2(dx, dx, fma2(dy, dy, nhi));
                sure |= lo32(zl) | hi32(zl);
                maybe |= lo32(zh) | hi32(zh);
            }
            for (uint32_t m = more23; m; m &= m - 1) {
                const int c = __ffs(m) - 1;
                const double2* p = reinterpret_cast<const double2*>(cell_at(cells, nbh.index(g, c, hx, hy)));
                const double2 x23 = __ldg(p + 1), y23 = __ldg(p + 3);
                const float sx = (float)dir_dx(c) * wxf, sy = (float)dir_dy(c) * wyf;
                const f2x dx = sub2(tx2, add2(pk(approx_f32(x23.x), approx_f32(x23.y)), pk(sx, sx)));
                const f2x dy = sub2(ty2, add2(pk(approx_f32(y23.x), approx_f32(y23.y)), pk(sy, sy)));
                const f2x zl = fma2(dx, dx, fma2(dy, dy, nlo)), zh = fma2(dx, dx, fma2(dy, dy, nhi));
                sure |= lo32(zl) | hi32(zl);
                maybe |= lo32(zh) | hi32(zh);
            }
            bool hit = (sure & 0x80000000u) != 0;
            if (inside && !hit && (maybe & 0x80000000u))
                hit = exact_trial_hit(g, cells, nbh, hx, hy, own, ofx, ofy, i, tx, ty, txf, tyf);
            const bool ok = inside && !hit;
            put_if(own.x, i, tx, ok);
            put_if(own.y, i, ty, ok);
            put_if(ofx, i, txf, ok);
            put_if(ofy, i, tyf, ok);
            ++n_tr;
            n_acc += ok;
            n_leave += !inside;
            i = (i + 1 == n) ? 0 : i + 1;
        }
        store_cell(ownp, own);
    }
    add_block_counters<ROWS>(n_tr, n_acc, n_leave, bpart);
}

// One-warp blocks (one set row of 32 cells), 16 per SM (128 registers).
static __global__ void __launch_bounds__(32, 16)
k_subsweep_f64(const Geometry g, double* __restrict__ cells, const SweepDraw* __restrict__ draw, int k,
               unsigned long long* __restrict__ partial) {
    pdl_release();
    pdl_wait();
    // counters of the tile that holds this block (shared: atomic adds)
    subsweep_f64<1>(g, cells, draw, k, blockIdx.x, blockIdx.y,
                    partial + 4 * ((long long)(blockIdx.y / kCounterRows) * gridDim.x + blockIdx.x));
}

}  // namespace hdmc
