// hdmc_kernels.cuh -- sub-sweep, cell-shift and contact-histogram kernels.
// Included once by each precision's translation unit.
//
// Cell storage (per cell, 4 slots): x0 x1 x2 x3 y0 y1 y2 y3 in the coordinate
// type (32 B for binary32, 64 B for binary64); an unused slot holds kEmpty.
// The cells of one checkerboard set are contiguous (see storage_index).
//
// Every floating-point operation that decides an acceptance, an ownership or
// a histogram bin is written with an explicit round-to-nearest operation, so
// the result does not depend on compiler contraction:
//   binary64: trial coordinate p + d*u, overlap iff dx*dx + dy*dy < sigma^2;
//   binary32: trial coordinate fma(d, u, p), overlap iff
//             fma(dx, dx, fma(dy, dy, -sigma^2)) < 0.
#pragma once

#include <utility>

#include "hdmc_device.cuh"

namespace hdmc {

constexpr int kDirChunk = 8;   // trial directions drawn ahead per thread (binary32 sub-sweep)

// ---- packed binary32 pairs (Blackwell f32x2 arithmetic, IEEE round-to-nearest per lane) ----
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk(float lo, float hi) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ uint32_t lo32(f2x v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t hi32(f2x v) { return (uint32_t)(v >> 32); }

// z = fma(dx, dx, fma(dy, dy, -sigma^2)) for two candidates at once; the sign
// bit of each half is set iff that candidate overlaps the trial position.
__device__ __forceinline__ f2x zpair(f2x tx2, f2x ty2, f2x qx2, f2x qy2, f2x ns2) {
    const f2x dx = sub2(tx2, qx2);
    const f2x dy = sub2(ty2, qy2);
    return fma2(dx, dx, fma2(dy, dy, ns2));
}

// ---- 21-bit fields of a Philox block (binary32 draws) -------------------------
// Field j = bits [21j, 21j+21) of the 128-bit integer w.x + 2^32 w.y + 2^64 w.z + 2^96 w.w.
__device__ __forceinline__ void fields21(const uint4 w, uint32_t f[6]) {
    const uint32_t M = 0x1FFFFFu;
    f[0] = w.x & M;
    f[1] = __funnelshift_r(w.x, w.y, 21) & M;
    f[2] = (w.y >> 10) & M;
    f[3] = __funnelshift_r(w.y, w.z, 31) & M;
    f[4] = __funnelshift_r(w.z, w.w, 20) & M;
    f[5] = (w.w >> 9) & M;
}
// Odd multiples of 2^-21 in (-1,1).
__device__ __forceinline__ float sym21(uint32_t f) {
    return (float)((int32_t)(2 * f + 1) - (1 << 21)) * 0x1p-21f;
}


__device__ __forceinline__ uint32_t factorial(int n) { return n == 4 ? 24u : n == 3 ? 6u : n == 2 ? 2u : 1u; }

// ---- cells ---------------------------------------------------------------------
template <typename T> struct Cell { T x[4], y[4]; };

__device__ __forceinline__ void load_cell(const float* p, Cell<float>& c) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    c.x[0] = a.x; c.x[1] = a.y; c.x[2] = a.z; c.x[3] = a.w;
    c.y[0] = b.x; c.y[1] = b.y; c.y[2] = b.z; c.y[3] = b.w;
}
__device__ __forceinline__ void load_cell_ro(const float* p, Cell<float>& c) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    c.x[0] = a.x; c.x[1] = a.y; c.x[2] = a.z; c.x[3] = a.w;
    c.y[0] = b.x; c.y[1] = b.y; c.y[2] = b.z; c.y[3] = b.w;
}
__device__ __forceinline__ void store_cell(float* p, const Cell<float>& c) {
    reinterpret_cast<float4*>(p)[0] = make_float4(c.x[0], c.x[1], c.x[2], c.x[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(c.y[0], c.y[1], c.y[2], c.y[3]);
}
__device__ __forceinline__ void load_cell(const double* p, Cell<double>& c) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = q[0], b = q[1], e = q[2], f = q[3];
    c.x[0] = a.x; c.x[1] = a.y; c.x[2] = b.x; c.x[3] = b.y;
    c.y[0] = e.x; c.y[1] = e.y; c.y[2] = f.x; c.y[3] = f.y;
}
__device__ __forceinline__ void load_cell_ro(const double* p, Cell<double>& c) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldg(q), b = __ldg(q + 1), e = __ldg(q + 2), f = __ldg(q + 3);
    c.x[0] = a.x; c.x[1] = a.y; c.x[2] = b.x; c.x[3] = b.y;
    c.y[0] = e.x; c.y[1] = e.y; c.y[2] = f.x; c.y[3] = f.y;
}
__device__ __forceinline__ void store_cell(double* p, const Cell<double>& c) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(c.x[0], c.x[1]);
    q[1] = make_double2(c.x[2], c.x[3]);
    q[2] = make_double2(c.y[0], c.y[1]);
    q[3] = make_double2(c.y[2], c.y[3]);
}

template <typename T>
__device__ __forceinline__ T pick(const T a[4], int i) {
    return i == 0 ? a[0] : i == 1 ? a[1] : i == 2 ? a[2] : a[3];
}
template <typename T>
__device__ __forceinline__ void put_if(T a[4], int i, T v, bool p) {
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = (p && i == j) ? v : a[j];
}

// pick / put_if when i is known to lie in the slot set M (bit j = slot j).
template <unsigned M, typename T>
__device__ __forceinline__ T pick_in(const T a[4], int i) {
    constexpr int top = (M & 8u) ? 3 : (M & 4u) ? 2 : (M & 2u) ? 1 : 0;
    T r = a[top];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j != top && ((M >> j) & 1u)) r = (i == j) ? a[j] : r;
    return r;
}
template <unsigned M, typename T>
__device__ __forceinline__ void put_in(T a[4], int i, T v, bool p) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if ((M >> j) & 1u) a[j] = (p && i == j) ? v : a[j];
}

// Slots that trial t can visit when the n <= 4 disks are visited cyclically
// from slot 0: {t mod n : n = 1..4}.
__host__ __device__ constexpr unsigned trial_slots(int t) {
    return (1u << (t % 1)) | (1u << (t % 2)) | (1u << (t % 3)) | (1u << (t % 4));
}
template <typename F, int... T>
__device__ __forceinline__ void unrolled_trials(F& f, std::integer_sequence<int, T...>) {
    (f(T, std::integral_constant<unsigned, trial_slots(T)>{}), ...);
}
// Swap slot J (compile time) with slot s <= J of both coordinate arrays.
template <int J, typename T>
__device__ __forceinline__ void swap_slot(T x[4], T y[4], int s) {
    T xs = x[J], ys = y[J];
#pragma unroll
    for (int m = 0; m < J; ++m) {
        xs = s == m ? x[m] : xs;
        ys = s == m ? y[m] : ys;
    }
    const T xj = x[J], yj = y[J];
#pragma unroll
    for (int m = 0; m < J; ++m) {
        x[m] = s == m ? xj : x[m];
        y[m] = s == m ? yj : y[m];
    }
    x[J] = xs;
    y[J] = ys;
}

// Uniform shuffle of the n <= 4 occupied slots (Alg. 1, the disks of a cell)
// from one draw k in [0, n!): Fisher-Yates swaps of slot j with slot
// k mod (j+1), k /= (j+1), for j = n-1 down to 1, applied to the
// coordinates in place (a swap whose j is not below n is skipped).
template <typename T>
__device__ __forceinline__ void shuffle_slots(T x[4], T y[4], int n, uint32_t k) {
    const int s3 = n >= 4 ? (int)(k & 3u) : 3;
    const uint32_t k1 = n >= 4 ? k >> 2 : k;
    const int s2 = n >= 3 ? (int)(k1 % 3u) : 2;
    const uint32_t k2 = n >= 3 ? k1 / 3u : k1;
    const int s1 = n >= 2 ? (int)(k2 & 1u) : 1;
    swap_slot<3>(x, y, s3);
    swap_slot<2>(x, y, s2);
    swap_slot<1>(x, y, s1);
}

__device__ __forceinline__ int wrap(int c, int m) { return c < 0 ? c + m : (c >= m ? c - m : c); }

// Truncating binary64 -> binary32 with integer instructions only (relative
// error < 2^-23; magnitudes below 2^-126 become 0).  Used for conservative
// prefilters, never for a decision.
__device__ __forceinline__ float approx_f32(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return e < 897u ? __uint_as_float(hi & 0x80000000u) : __uint_as_float(f);
}

// Per-block trial counters: bpart[{trials, accepted, left, overlap}] of this
// block's own slot (blocks with the same slot run in stream order, so the
// read-modify-write needs no atomics).
template <int ROWS>
__device__ __forceinline__ void add_block_counters(unsigned int n_tr, unsigned int n_acc, unsigned int n_leave,
                                                   unsigned long long* __restrict__ bpart) {
    __shared__ unsigned int red[ROWS][3];
    const unsigned a = __reduce_add_sync(0xffffffffu, n_tr);
    const unsigned b = __reduce_add_sync(0xffffffffu, n_acc);
    const unsigned c = __reduce_add_sync(0xffffffffu, n_leave);
    if (threadIdx.x == 0) {
        red[threadIdx.y][0] = a;
        red[threadIdx.y][1] = b;
        red[threadIdx.y][2] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        unsigned tr = 0, ac = 0, lv = 0;
#pragma unroll
        for (int w = 0; w < ROWS; ++w) {
            tr += red[w][0];
            ac += red[w][1];
            lv += red[w][2];
        }
        bpart[0] += tr;
        bpart[1] += ac;
        bpart[2] += lv;
        bpart[3] += tr - ac - lv;
    }
}

// ---- neighbourhood of an active cell on the set-major layout ---------------------------
// For a cell of set Q = qx + 2 qy at half-grid position (hx, hy), the
// neighbours (cx +- 1, cy) lie in set Q^1 at half-columns xl, xr, the
// neighbours (cx, cy +- 1) in set Q^2 at half-rows yd, yu, the diagonal ones
// in set Q^3 (periodic wrap on the half grid).  Directions c = 0..7 run over
// (dx,dy) = (-1,-1) (0,-1) (1,-1) (-1,0) (1,0) (-1,1) (0,1) (1,1).
// Cell indices are 32-bit here (the grid has fewer than 2^32 cells) and are
// widened once, in cell_at.
struct Neighbourhood {
    uint32_t base[4];   // first cell of set Q, Q^1, Q^2, Q^3
    int xl, xr, yd, yu;
    __device__ Neighbourhood(const Geometry& g, int Q, int hx, int hy) {
        const int qx = Q & 1, qy = Q >> 1;
        const uint32_t cq = (uint32_t)g.cq;
        base[0] = (uint32_t)Q * cq;
        base[1] = (uint32_t)(Q ^ 1) * cq;
        base[2] = (uint32_t)(Q ^ 2) * cq;
        base[3] = (uint32_t)(Q ^ 3) * cq;
        xl = hx - 1 + qx;
        xl = xl < 0 ? g.hx - 1 : xl;
        xr = hx + qx;
        xr = xr >= g.hx ? 0 : xr;
        yd = hy - 1 + qy;
        yd = yd < 0 ? g.hy - 1 : yd;
        yu = hy + qy;
        yu = yu >= g.hy ? 0 : yu;
    }
    __device__ __forceinline__ uint32_t index(const Geometry& g, int c, int hx, int hy) const {
        const int col = (c == 1 || c == 6) ? hx : ((c == 0 || c == 3 || c == 5) ? xl : xr);
        const int row = (c < 3) ? yd : (c < 5 ? hy : yu);
        const int set = (c == 3 || c == 4) ? 1 : ((c == 1 || c == 6) ? 2 : 3);
        return base[set] + (uint32_t)row * (uint32_t)g.hx + (uint32_t)col;
    }
    __device__ __forceinline__ uint32_t own(const Geometry& g, int hx, int hy) const {
        return base[0] + (uint32_t)hy * (uint32_t)g.hx + (uint32_t)hx;
    }
};
template <typename T>
__device__ __forceinline__ T* cell_at(T* cells, uint32_t idx) {
    return cells + 8 * (size_t)idx;
}
__device__ __forceinline__ int dir_dx(int c) { return (c == 1 || c == 6) ? 0 : ((c == 0 || c == 3 || c == 5) ? -1 : 1); }
__device__ __forceinline__ int dir_dy(int c) { return c < 3 ? -1 : (c < 5 ? 0 : 1); }

// ---- binary32 sub-sweep: Alg. 1 lines 4-13 / Alg. 2 ----------------------------------
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

template <int ROWS, int NSEL, bool TRACK = false>
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
    const bool live = hx < g.hx && hy < g.hy;
    const int cx = 2 * hx + (Q & 1), cy = 2 * hy + (Q >> 1);
    const Neighbourhood nbh(g, Q, hx, hy);

    // 1. loads
    Cell<float> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = (float)kEmpty;
    float* ownp = cell_at(cells, nbh.own(g, hx, hy));
    if (live) load_cell(ownp, own);
    float4 n01[8];   // slots 0,1 of the neighbours (x0 x1 y0 y1); slot 2 only to flag its use
    float n2[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        n01[c] = make_float4((float)kEmpty, (float)kEmpty, (float)kEmpty, (float)kEmpty);
        n2[c] = (float)kEmpty;
        if (live) {
            const float* p = cell_at(cells, nbh.index(g, c, hx, hy));
            const float2 x01 = __ldg(reinterpret_cast<const float2*>(p));
            const float2 y01 = __ldg(reinterpret_cast<const float2*>(p) + 2);
            n01[c] = make_float4(x01.x, x01.y, y01.x, y01.y);
            n2[c] = __ldg(p + 2);
        }
    }

    // 2. directions of the first chunk (the cell's trial stream)
    const uint32_t cell = (uint32_t)cy * (uint32_t)g.mx + (uint32_t)cx;
    const uint32_t c2 = (kDomTrial << 28) | ((uint32_t)Q << 24);
    uint32_t F[6];
    fields21(philox4x32_10(make_uint4(sweep, cell, c2, 0u), g.key0, g.key1), F);
    const uint32_t f0 = F[0];   // shuffle draw
    uint32_t blk = 0;
    int pnext = 1;               // next attempt: field pair 1 of block 0 (fields 2,3)
    draw_directions<ROWS>(g, sweep, cell, c2, F, blk, pnext, min(kDirChunk, nsel), sdir, tid);

    // 3. cell contents
    const int n = (own.x[0] >= 0.f) + (own.x[1] >= 0.f) + (own.x[2] >= 0.f) + (own.x[3] >= 0.f);
    uint32_t dir23 = 0;   // warp-uniform: directions where some lane has a third disk
#pragma unroll
    for (int c = 0; c < 8; ++c) dir23 |= __any_sync(0xffffffffu, n2[c] >= 0.f) ? (1u << c) : 0u;
    const bool own23 = __any_sync(0xffffffffu, n >= 3);

    unsigned int n_tr = 0, n_acc = 0, n_leave = 0;
    float net2 = 0.f;
    if (n > 0) {
        // shuffle (Alg. 1 line 5): one draw in [0, n!) by 21-bit Lemire on field 0
        if (n >= 2) {
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
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float sx = (float)dir_dx(c) * g.wxf, sy = (float)dir_dy(c) * g.wyf;
            qx01[c] = add2(pk(n01[c].x, n01[c].y), pk(sx, sx));
            qy01[c] = add2(pk(n01[c].z, n01[c].w), pk(sy, sy));
        }
        // slot pair (2,3) of the first flagged direction, translated; further
        // flagged directions (rare) are read in the trial loop
        f2x fx23 = 0, fy23 = 0;
        const uint32_t more23 = dir23 & (dir23 - 1);
        if (dir23) {
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
                if (own23) {
                    z = zpair(tx2, ty2, pk(own.x[2], own.x[3]), pk(own.y[2], own.y[3]), ns2);
                    acc |= ((M & 4u) && i == 2 ? 0u : lo32(z)) | ((M & 8u) && i == 3 ? 0u : hi32(z));
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    z = zpair(tx2, ty2, qx01[c], qy01[c], ns2);
                    acc |= lo32(z) | hi32(z);
                }
                if (dir23) {
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

template <int ROWS, int NSEL>
static __global__ void __launch_bounds__(32 * ROWS, 20 / ROWS)
k_subsweep_f32(const Geometry g, float* __restrict__ cells, const SweepDraw* __restrict__ draw, int k,
               unsigned long long* __restrict__ partial) {
    __shared__ float2 sdir[kDirChunk][32 * ROWS];
    subsweep_f32<ROWS, NSEL>(g, cells, draw, k, blockIdx.x, blockIdx.y,
                             partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x), sdir);
}

// Coordinate-type helpers: widths, shift distance, next value below w,
// explicitly rounded add/sub, exact comparisons.
template <typename T> struct Prm;
template <> struct Prm<float> {
    static __device__ __forceinline__ float wx(const Geometry& g) { return g.wxf; }
    static __device__ __forceinline__ float wy(const Geometry& g) { return g.wyf; }
    static __device__ __forceinline__ float ds(const SweepDraw& r) { return r.dsf; }
    static __device__ __forceinline__ float prev(float w) { return __uint_as_float(__float_as_uint(w) - 1u); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ bool ge0(float x) { return x >= 0.f; }
    static __device__ __forceinline__ bool lt(float x, float w) { return x < w; }
};
template <> struct Prm<double> {
    static __device__ __forceinline__ double wx(const Geometry& g) { return g.wx; }
    static __device__ __forceinline__ double wy(const Geometry& g) { return g.wy; }
    static __device__ __forceinline__ double ds(const SweepDraw& r) { return r.ds; }
    static __device__ __forceinline__ double prev(double w) {
        return __longlong_as_double(__double_as_longlong(w) - 1ll);
    }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    // Comparisons on the integer pipe (binary64 ones are slow on this GPU);
    // exact for every non-NaN x: ge0(x) == (x >= 0) (the bit patterns of
    // +0 .. +inf and of -0 are at most 2^63 unsigned), and for w > 0
    // lt(x, w) == (x < w) (negative x read as a negative integer).
    static __device__ __forceinline__ bool ge0(double x) {
        return (unsigned long long)__double_as_longlong(x) <= 0x8000000000000000ull;
    }
    static __device__ __forceinline__ bool lt(double x, double w) {
        return __double_as_longlong(x) < __double_as_longlong(w);
    }
};

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

__device__ __forceinline__ void subsweep_f64(const Geometry& g, double* __restrict__ cells,
                                             const SweepDraw* __restrict__ draw, int k, int bx, int by,
                                             unsigned long long* __restrict__ bpart) {
    const int Q = draw->perm[k];
    const uint32_t sweep = draw->sweep;
    const int hx = bx * 32 + threadIdx.x;
    const int hy = by * 4 + threadIdx.y;
    const bool live = hx < g.hx && hy < g.hy;
    const int cx = 2 * hx + (Q & 1), cy = 2 * hy + (Q >> 1);
    const Neighbourhood nbh(g, Q, hx, hy);

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
        const uint32_t cell = (uint32_t)cy * (uint32_t)g.mx + (uint32_t)cx;
        const uint32_t setbits = (uint32_t)Q << 24;
        if (n >= 2) {
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
    add_block_counters<4>(n_tr, n_acc, n_leave, bpart);
}

static __global__ void __launch_bounds__(128, 3)
k_subsweep_f64(const Geometry g, double* __restrict__ cells, const SweepDraw* __restrict__ draw, int k,
               unsigned long long* __restrict__ partial) {
    subsweep_f64(g, cells, draw, k, blockIdx.x, blockIdx.y,
                 partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x));
}


// ---- cell shift: Alg. 4 ----------------------------------------------------------------
// One thread per new cell; grid (set row, set column, set).  New cell c = the
// disks of old c that stay inside c after the translation by -f*ds (old slot
// order), then the disks of old c+f that leave c+f, re-expressed in c's frame
// (+f*w).  The ownership test is the same expression in the two threads that
// see a disk, so every disk lands in exactly one cell (Sec. 3.2).  A
// re-expressed value that rounds onto the upper edge is clamped below it.
template <typename T>
__device__ __forceinline__ void shift_cells(const Geometry& g, const T* __restrict__ src, T* __restrict__ dst,
                                            const SweepDraw* __restrict__ draw, DevState* __restrict__ st, int bx,
                                            int by, int q) {
    const int hx = bx * kShiftBX + threadIdx.x;
    const int hy = by * kShiftBY + threadIdx.y;
    const int fdir = draw->fdir;
    const int ax = fdir >> 1;
    const int sgn = (fdir & 1) ? -1 : 1;
    const T w = ax ? Prm<T>::wy(g) : Prm<T>::wx(g);
    const T sd = T(sgn) * Prm<T>::ds(*draw);
    const T sw = T(sgn) * w;
    if (hx == 0 && hy == 0 && q == 0) st->origin[ax] += (double)sd;
    if (hx >= g.hx || hy >= g.hy) return;
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    const int ncx = ax ? cx : wrap(cx + sgn, g.mx);
    const int ncy = ax ? wrap(cy + sgn, g.my) : cy;
    const long long idx = (long long)q * g.cq + (long long)hy * g.hx + hx;
    Cell<T> o, b, r;
    load_cell_ro(src + 8 * idx, o);
    load_cell_ro(src + 8 * storage_index(g, ncx, ncy), b);
#pragma unroll
    for (int j = 0; j < 4; ++j) r.x[j] = r.y[j] = T(kEmpty);
    int kept = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (Prm<T>::ge0(o.x[j])) {
            const T dp = Prm<T>::sub(ax ? o.y[j] : o.x[j], sd);
            if (Prm<T>::ge0(dp) && Prm<T>::lt(dp, w)) {
                const T vx = ax ? o.x[j] : dp, vy = ax ? dp : o.y[j];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    r.x[s] = (kept == s) ? vx : r.x[s];
                    r.y[s] = (kept == s) ? vy : r.y[s];
                }
                ++kept;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (Prm<T>::ge0(b.x[j])) {
            const T dp = Prm<T>::sub(ax ? b.y[j] : b.x[j], sd);
            if (!(Prm<T>::ge0(dp) && Prm<T>::lt(dp, w))) {
                T v = Prm<T>::add(dp, sw);
                v = Prm<T>::lt(v, w) ? v : Prm<T>::prev(w);
                v = Prm<T>::ge0(v) ? v : T(0);
                const T vx = ax ? b.x[j] : v, vy = ax ? v : b.y[j];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    r.x[s] = (kept == s) ? vx : r.x[s];
                    r.y[s] = (kept == s) ? vy : r.y[s];
                }
                ++kept;
            }
        }
    }
    if (kept > 4) atomicOr(&st->error, 1u);
    store_cell(dst + 8 * idx, r);
}

template <typename T>
__global__ void __launch_bounds__(kShiftBX * kShiftBY)
k_shift(const Geometry g, const T* __restrict__ src, T* __restrict__ dst, const SweepDraw* __restrict__ draw,
        DevState* __restrict__ st) {
    shift_cells<T>(g, src, dst, draw, st, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---- contact histogram: Sec. 4 ------------------------------------------------------
// Ordered pairs (i, j != i) at distance r in [sigma, sigma + 200 dr), in bins
// [sigma + b dr, sigma + (b+1) dr) decided on the binary64 r^2 against the
// squared bin edges; distances from cell-local coordinates over the 5x5
// neighbourhood (w >= sigma, so two rings reach past 1.02 sigma).  A binary32
// estimate of r^2 with a wide margin selects the candidates (about 0.7 per
// disk); each warp queues its candidates in shared memory and computes the
// binary64 distance and bin of 32 queued pairs at a time, so the (slow)
// binary64 instructions run with every lane busy.  Non-negative doubles
// order like their bit patterns read as signed integers, so the bin search
// compares integers.  One thread per cell, grid (set row, set column, set);
// per-block shared histogram.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return approx_f32(v); }

constexpr int kHistQueue = 64;   // per-warp candidate queue (< 32 pending + 32 appended)

// Candidate entry: source lane (5 bits), own slot i (2), neighbour slot j (2),
// dx + 2 (3), dy + 2 (3).
__device__ __forceinline__ uint32_t hist_entry(int lane, int b, int dx, int dy) {
    return (uint32_t)lane | ((uint32_t)(b >> 2) << 5) | ((uint32_t)(b & 3) << 7) | ((uint32_t)(dx + 2) << 9) |
           ((uint32_t)(dy + 2) << 12);
}

// Bins the first `count` queued pairs, one per lane (warp-uniform call).
template <typename T>
__device__ __forceinline__ void hist_flush(const Geometry& g, const T* __restrict__ cells, const uint32_t* sq,
                                           int count, int q, int bx, int hy, const long long* sEi,
                                           unsigned int* sh, double wxd, double wyd, float sigf, float inv_drf) {
    const int lane = threadIdx.x;
    if (lane >= count) return;
    const uint32_t e = sq[lane];
    const int src = e & 31, i = (e >> 5) & 3, j = (e >> 7) & 3;
    const int dx = (int)((e >> 9) & 7) - 2, dy = (int)((e >> 12) & 7) - 2;
    const int hx = bx * kHistBX + src;
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    const T* own = cells + 8 * ((long long)q * g.cq + (long long)hy * g.hx + hx);
    const T* nb = cells + 8 * storage_index(g, wrap(cx + dx, g.mx), wrap(cy + dy, g.my));
    const double px = (double)__ldg(own + i), py = (double)__ldg(own + 4 + i);
    const double ex = __dadd_rn((double)__ldg(nb + j), (double)dx * wxd);
    const double ey = __dadd_rn((double)__ldg(nb + 4 + j), (double)dy * wyd);
    const double ddx = __dsub_rn(px, ex), ddy = __dsub_rn(py, ey);
    const double r2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
    const long long r2i = __double_as_longlong(r2);   // r2 >= +0
    if (r2i >= sEi[0] && r2i < sEi[kHistBins]) {
        // bin b: sE[b] <= r2 < sE[b+1]; start from a binary32 estimate
        const float r2f = approx_f32(r2);
        int bb = (int)((r2f * rsqrtf(r2f) - sigf) * inv_drf);
        bb = bb < 0 ? 0 : (bb > kHistBins - 1 ? kHistBins - 1 : bb);
        while (bb > 0 && r2i < sEi[bb]) --bb;
        while (bb < kHistBins - 1 && r2i >= sEi[bb + 1]) ++bb;
        atomicAdd(&sh[bb], 1u);
    }
}

template <typename T>
__device__ __forceinline__ void hist_cells(const Geometry& g, const T* __restrict__ cells,
                                           const double* __restrict__ edges2, unsigned long long* __restrict__ hist,
                                           int bx, int by, int q) {
    __shared__ unsigned int sh[kHistBins];
    __shared__ long long sEi[kHistBins + 1];   // bit patterns of the squared edges
    __shared__ uint32_t squeue[kHistBY][kHistQueue];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int b = tid; b < kHistBins; b += blockDim.x * blockDim.y) sh[b] = 0u;
    for (int b = tid; b <= kHistBins; b += blockDim.x * blockDim.y) sEi[b] = __double_as_longlong(edges2[b]);
    __syncthreads();
    const int lane = threadIdx.x;
    const int hx = bx * kHistBX + threadIdx.x;
    const int hy = by * kHistBY + threadIdx.y;
    const bool live = hx < g.hx && hy < g.hy;
    uint32_t* sq = squeue[threadIdx.y];
    Cell<T> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = T(kEmpty);
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    if (live) load_cell_ro(cells + 8 * ((long long)q * g.cq + (long long)hy * g.hx + hx), own);
    const bool any = __any_sync(0xffffffffu, Prm<T>::ge0(own.x[0]));
    const bool own23 = __any_sync(0xffffffffu, Prm<T>::ge0(own.x[2]));
    if (any) {
        const double wxd = (double)Prm<T>::wx(g), wyd = (double)Prm<T>::wy(g);
        const float wxf = (float)Prm<T>::wx(g), wyf = (float)Prm<T>::wy(g);
        const float sigf = (float)g.sigma, inv_drf = (float)(1.0 / (kHistDr * g.sigma));
        const float rmax = (float)(g.sigma + kHistBins * kHistDr * g.sigma);
        const float thr = rmax * rmax * 1.001f;   // binary32 estimate margin (estimate error < 1e-6)
        float ox[4], oy[4];
        uint32_t occupied = 0;   // bits 4i..4i+3 set when own slot i holds a disk
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ox[i] = to_f32(own.x[i]);
            oy[i] = to_f32(own.y[i]);
            occupied |= Prm<T>::ge0(own.x[i]) ? (0xFu << (4 * i)) : 0u;
        }
        int qn = 0;   // queued candidates of this warp (warp-uniform)
        for (int dy = -2; dy <= 2; ++dy) {
            for (int dx = -2; dx <= 2; ++dx) {
                Cell<T> c;
#pragma unroll
                for (int j = 0; j < 4; ++j) c.x[j] = c.y[j] = T(kEmpty);
                if (live) load_cell_ro(cells + 8 * storage_index(g, wrap(cx + dx, g.mx), wrap(cy + dy, g.my)), c);
                const float sxf = (float)dx * wxf, syf = (float)dy * wyf;
                const f2x qx01 = add2(pk(to_f32(c.x[0]), to_f32(c.x[1])), pk(sxf, sxf));
                const f2x qx23 = add2(pk(to_f32(c.x[2]), to_f32(c.x[3])), pk(sxf, sxf));
                const f2x qy01 = add2(pk(to_f32(c.y[0]), to_f32(c.y[1])), pk(syf, syf));
                const f2x qy23 = add2(pk(to_f32(c.y[2]), to_f32(c.y[3])), pk(syf, syf));
                const f2x nt = pk(-thr, -thr);
                const bool c23 = __any_sync(0xffffffffu, Prm<T>::ge0(c.x[2]));
                uint32_t cand = 0;   // bit 4i+j: pair (own i, neighbour slot j) passes the estimate
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= 2 && !own23) continue;
                    const f2x tx2 = pk(ox[i], ox[i]), ty2 = pk(oy[i], oy[i]);
                    f2x z = zpair(tx2, ty2, qx01, qy01, nt);
                    cand |= ((lo32(z) >> 31) << (4 * i)) | ((hi32(z) >> 31) << (4 * i + 1));
                    if (c23) {
                        z = zpair(tx2, ty2, qx23, qy23, nt);
                        cand |= ((lo32(z) >> 31) << (4 * i + 2)) | ((hi32(z) >> 31) << (4 * i + 3));
                    }
                }
                // empty own slots are excluded (two empty slots sit one cell offset
                // apart), and no disk is paired with itself
                cand &= occupied;
                if (dx == 0 && dy == 0) cand &= ~0x8421u;
                for (;;) {   // queue the candidates, one per lane and round
                    const unsigned act = __ballot_sync(0xffffffffu, cand != 0);
                    if (!act) break;
                    if (cand) {
                        const int b = __ffs(cand) - 1;
                        cand &= cand - 1;
                        sq[qn + __popc(act & ((1u << lane) - 1u))] = hist_entry(lane, b, dx, dy);
                    }
                    qn += __popc(act);
                    if (qn >= 32) {
                        __syncwarp();
                        hist_flush<T>(g, cells, sq, 32, q, bx, hy, sEi, sh, wxd, wyd, sigf, inv_drf);
                        __syncwarp();
                        const uint32_t v = lane < qn - 32 ? sq[32 + lane] : 0u;
                        __syncwarp();
                        if (lane < qn - 32) sq[lane] = v;
                        __syncwarp();
                        qn -= 32;
                    }
                }
            }
        }
        __syncwarp();
        hist_flush<T>(g, cells, sq, qn, q, bx, hy, sEi, sh, wxd, wyd, sigf, inv_drf);
    }
    __syncthreads();
    for (int b = tid; b < kHistBins; b += blockDim.x * blockDim.y)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

template <typename T>
__global__ void __launch_bounds__(kHistBX * kHistBY)
k_hist(const Geometry g, const T* __restrict__ cells, const double* __restrict__ edges2,
       unsigned long long* __restrict__ hist) {
    hist_cells<T>(g, cells, edges2, hist, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---- batched replicas ------------------------------------------------------------------
// Every stage is one launch over all replicas of a batch: the launch's flat
// block index is mapped to (replica, local block) by a per-stage table, and
// each replica keeps its own geometry, cells, draws, device state,
// counters and histogram.  Replica r's cells start at cell rd.cell_off of
// the arena; its sweep draws of chunk position j sit at draws[j*R + r].
template <int ROWS, bool TRACK>
static __global__ void __launch_bounds__(32 * ROWS, 20 / ROWS)
k_subsweep_f32_batch(const ReplicaDesc* __restrict__ reps, const unsigned short* __restrict__ map,
                     float* __restrict__ arena, const SweepDraw* __restrict__ draws, int R, int j, int k,
                     unsigned long long* __restrict__ partial, double* __restrict__ msd) {
    __shared__ float2 sdir[kDirChunk][32 * ROWS];
    const int r = map[blockIdx.x];
    const ReplicaDesc* rd = reps + r;
    const int local = (int)blockIdx.x - rd->sub_block0;
    const int by = local / rd->sub_gx, bx = local - by * rd->sub_gx;
    subsweep_f32<ROWS, 0, TRACK>(rd->g, arena + 8 * rd->cell_off, draws + (size_t)j * R + r, k, bx, by,
                              partial + 4 * (rd->part_off + local), sdir, msd + r);
}

static __global__ void __launch_bounds__(128, 3)
k_subsweep_f64_batch(const ReplicaDesc* __restrict__ reps, const unsigned short* __restrict__ map,
                     double* __restrict__ arena, const SweepDraw* __restrict__ draws, int R, int j, int k,
                     unsigned long long* __restrict__ partial) {
    const int r = map[blockIdx.x];
    const ReplicaDesc* rd = reps + r;
    const int local = (int)blockIdx.x - rd->sub_block0;
    const int by = local / rd->sub_gx, bx = local - by * rd->sub_gx;
    subsweep_f64(rd->g, arena + 8 * rd->cell_off, draws + (size_t)j * R + r, k, bx, by,
                 partial + 4 * (rd->part_off + local));
}

template <typename T>
__global__ void __launch_bounds__(kShiftBX * kShiftBY)
k_shift_batch(const ReplicaDesc* __restrict__ reps, const unsigned short* __restrict__ map,
              const T* __restrict__ src, T* __restrict__ dst, const SweepDraw* __restrict__ draws, int R, int j,
              DevState* __restrict__ sts) {
    const int r = map[blockIdx.x];
    const ReplicaDesc* rd = reps + r;
    const int local = (int)blockIdx.x - rd->sh_block0;
    const int per_set = rd->sh_gx * rd->sh_gy;
    const int q = local / per_set, rem = local - q * per_set;
    const int by = rem / rd->sh_gx, bx = rem - by * rd->sh_gx;
    shift_cells<T>(rd->g, src + 8 * rd->cell_off, dst + 8 * rd->cell_off, draws + (size_t)j * R + r, sts + r, bx,
                   by, q);
}

template <typename T>
__global__ void __launch_bounds__(kHistBX * kHistBY)
k_hist_batch(const ReplicaDesc* __restrict__ reps, const unsigned short* __restrict__ map,
             const T* __restrict__ arena, const double* __restrict__ edges2, unsigned long long* __restrict__ hist) {
    const int r = map[blockIdx.x];
    const ReplicaDesc* rd = reps + r;
    const int local = (int)blockIdx.x - rd->hi_block0;
    const int per_set = rd->hi_gx * rd->hi_gy;
    const int q = local / per_set, rem = local - q * per_set;
    const int by = rem / rd->hi_gx, bx = rem - by * rd->hi_gx;
    hist_cells<T>(rd->g, arena + 8 * rd->cell_off, edges2, hist + (size_t)r * kHistBins, bx, by, q);
}

// ---- launchers ---------------------------------------------------------------------
inline dim3 set_grid(const Geometry& g, dim3 block) {
    return dim3((unsigned)((g.hx + block.x - 1) / block.x), (unsigned)((g.hy + block.y - 1) / block.y), 4u);
}

template <typename T>
void launch_shift_t(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw) {
    const dim3 block(kShiftBX, kShiftBY);
    k_shift<T><<<set_grid(c.g, block), block, 0, c.stream>>>(c.g, reinterpret_cast<const T*>(src),
                                                               reinterpret_cast<T*>(dst), draw, c.st);
}

template <typename T>
void launch_hist_t(const LaunchCtx& c, const void* cells) {
    const dim3 block(kHistBX, kHistBY);
    k_hist<T><<<set_grid(c.g, block), block, 0, c.stream>>>(c.g, reinterpret_cast<const T*>(cells), c.edges2,
                                                              c.hist);
}

// ---- snapshot check ---------------------------------------------------------------------
// Checks every cell of an incoming image (any storage order): occupied slots
// form a prefix, occupied coordinates lie in [0,wx) x [0,wy) of the
// coordinate type, unused slots hold kEmpty in both coordinates.  out[0]
// accumulates the number of disks, out[1] becomes non-zero on a bad cell.
template <typename T>
__global__ void __launch_bounds__(256) k_check_cells(const Geometry g, const T* __restrict__ cells,
                                                     unsigned long long* __restrict__ out) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    unsigned n = 0;
    bool bad = false;
    if (i < g.C) {
        Cell<T> c;
        load_cell_ro(cells + 8 * i, c);
        bool empty_seen = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (c.x[j] == T(kEmpty) && c.y[j] == T(kEmpty)) {
                empty_seen = true;
            } else {
                bad |= empty_seen || !(c.x[j] >= T(0) && c.x[j] < Prm<T>::wx(g)) ||
                       !(c.y[j] >= T(0) && c.y[j] < Prm<T>::wy(g));
                ++n;
            }
        }
    }
    const unsigned tot = __reduce_add_sync(0xffffffffu, n);
    if (threadIdx.x % 32 == 0 && tot) atomicAdd(out, (unsigned long long)tot);
    if (bad) atomicOr(out + 1, 1ull);
}

template <typename T>
void launch_check_t(const LaunchCtx& c, const void* cells, unsigned long long* out) {
    const unsigned blocks = (unsigned)((c.g.C + 255) / 256);
    k_check_cells<T><<<blocks, 256, 0, c.stream>>>(c.g, reinterpret_cast<const T*>(cells), out);
}

}  // namespace hdmc
