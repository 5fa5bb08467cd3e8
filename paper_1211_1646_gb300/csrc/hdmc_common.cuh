// hdmc_common.cuh -- device helpers shared by the kernels: packed binary32
// pairs, 21-bit random fields, cell loads and stores, slot selection and the
// in-cell shuffle, the checkerboard neighbourhood on the set-major layout,
// and the coordinate-type helpers.
//
// Cell storage (per cell, 4 slots): x0 x1 x2 x3 y0 y1 y2 y3 in the coordinate
// type (32 B for binary32, 64 B for binary64); an unused slot holds kEmpty.
// The cells of one checkerboard set are contiguous (see storage_index).
#pragma once

#include <utility>

#include "hdmc_device.cuh"

namespace hdmc {

// Programmatic dependent launch (launch_on with c.pdl): pdl_release lets the
// next kernel of the stream launch once every block of this grid has called
// it; pdl_wait returns when the previous kernel has completed and its writes
// are visible (at once for a normal launch).  Kernels launched this way call
// both before their first memory access.
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr int kDirChunk = 8;   // trial directions drawn ahead per thread (binary32 sub-sweep)
constexpr int kDirRows = kDirChunk + 2;   // rows of its buffer: a one-pass draw keeps up to two more

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
// Odd multiples of 2^-21 in (-1,1): (2f + 1 - 2^21) 2^-21, formed as
// 2 (1 + f 2^-21) - 3 + 2^-21 from the binary32 1 + f 2^-21 (f in the top
// of the significand); the FMA is exact, its result having 22 bits.
__device__ __forceinline__ float sym21(uint32_t f) {
    return __fmaf_rn(__uint_as_float(0x3F800000u | (f << 2)), 2.0f, -3.0f + 0x1p-21f);
}


__device__ __forceinline__ uint32_t factorial(int n) { return n == 4 ? 24u : n == 3 ? 6u : n == 2 ? 2u : 1u; }

// ---- cells ---------------------------------------------------------------------
template <typename T> struct Cell { T x[4], y[4]; };

// Whole binary32 cells with one 256-bit vector load or store (sm_100 and
// later); cells are 32-byte aligned (256-byte aligned buffers, 32-byte
// cells).  Binary64 cells use four 128-bit accesses, which measured faster
// in the binary64 kernels.
// The _ro loads take the read-only path: only for cells the kernel does
// not write.  The loads are volatile: each stays where it is written.
__device__ __forceinline__ void load_cell(const float* p, Cell<float>& c) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c.x[0]), "=f"(c.x[1]), "=f"(c.x[2]), "=f"(c.x[3]), "=f"(c.y[0]), "=f"(c.y[1]), "=f"(c.y[2]),
          "=f"(c.y[3])
        : "l"(p));
}
__device__ __forceinline__ void load_cell_ro(const float* p, Cell<float>& c) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c.x[0]), "=f"(c.x[1]), "=f"(c.x[2]), "=f"(c.x[3]), "=f"(c.y[0]), "=f"(c.y[1]), "=f"(c.y[2]),
          "=f"(c.y[3])
        : "l"(p));
}
__device__ __forceinline__ void store_cell(float* p, const Cell<float>& c) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(c.x[0]), "f"(c.x[1]),
                 "f"(c.x[2]), "f"(c.x[3]), "f"(c.y[0]), "f"(c.y[1]), "f"(c.y[2]), "f"(c.y[3])
                 : "memory");
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

// Per-block trial counters bpart[{trials, accepted, left, overlap}] of the
// block's own slot: each warp adds its sums with fire-and-forget atomic
// adds (no value returned, so nothing waits on the round trip; integer sums
// do not depend on their order).
template <int ROWS>
__device__ __forceinline__ void add_block_counters(unsigned int n_tr, unsigned int n_acc, unsigned int n_leave,
                                                   unsigned long long* __restrict__ bpart) {
    const unsigned a = __reduce_add_sync(0xffffffffu, n_tr);
    const unsigned b = __reduce_add_sync(0xffffffffu, n_acc);
    const unsigned c = __reduce_add_sync(0xffffffffu, n_leave);
    if (threadIdx.x == 0 && a != 0) {
        atomicAdd(bpart + 0, (unsigned long long)a);
        atomicAdd(bpart + 1, (unsigned long long)b);
        atomicAdd(bpart + 2, (unsigned long long)c);
        atomicAdd(bpart + 3, (unsigned long long)(a - b - c));
    }
}

// ---- neighbourhood of an active cell on the set-major layout ---------------------------
// For a cell of set Q = qx + 2 qy at half-grid position (hx, hy), the
// neighbours (cx +- 1, cy) lie in set Q^1 at half-columns xl, xr, the
// neighbours (cx, cy +- 1) in set Q^2 at half-rows yd, yu, the diagonal ones
// in set Q^3 (periodic wrap on the half grid).  Directions c = 0..7 run over
// (dx,dy) = (-1,-1) (0,-1) (1,-1) (-1,0) (1,0) (-1,1) (0,1) (1,1).
// Cell indices are 32-bit here (the grid has fewer than 2^32 cells) and are
// widened once, in cell_at.  Lanes past the end of a row (live = false)
// compute indices they never use; a -DHDMC_CHECK build checks the live ones.
struct Neighbourhood {
    uint32_t base[4];   // first cell of set Q, Q^1, Q^2, Q^3
    int xl, xr, yd, yu;
#ifdef HDMC_CHECK
    bool live;
#endif
    __device__ Neighbourhood(const Geometry& g, int Q, int hx, int hy, bool live_) {
#ifdef HDMC_CHECK
        live = live_;
#else
        (void)live_;
#endif
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
        // selects, not base[set]: a runtime index would put the array in local memory
        const uint32_t b = (c == 3 || c == 4) ? base[1] : ((c == 1 || c == 6) ? base[2] : base[3]);
        return checked(g, b + (uint32_t)row * (uint32_t)g.hx + (uint32_t)col);
    }
    __device__ __forceinline__ uint32_t own(const Geometry& g, int hx, int hy) const {
        return checked(g, base[0] + (uint32_t)hy * (uint32_t)g.hx + (uint32_t)hx);
    }
    __device__ __forceinline__ uint32_t checked(const Geometry& g, uint32_t i) const {
#ifdef HDMC_CHECK
        if (live) return (uint32_t)checked_cell(g.check, i, g.C);
#else
        (void)g;
#endif
        return i;
    }
};
template <typename T>
__device__ __forceinline__ T* cell_at(T* cells, uint32_t idx) {
    return cells + 8 * (size_t)idx;
}
__device__ __forceinline__ int dir_dx(int c) { return (c == 1 || c == 6) ? 0 : ((c == 0 || c == 3 || c == 5) ? -1 : 1); }
__device__ __forceinline__ int dir_dy(int c) { return c < 3 ? -1 : (c < 5 ? 0 : 1); }

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

}  // namespace hdmc
