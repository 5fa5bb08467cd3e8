// hdmc_kernels.cuh -- sub-sweep, cell-shift and contact-histogram kernels,
// templated on the coordinate type (double: HDMC_FP64, float:
// HDMC_FP32_LOCAL).  Included once by each precision's translation unit.
//
// Every floating-point operation that decides an acceptance, an ownership or
// a histogram bin is written with an explicit round-to-nearest intrinsic, so
// the result does not depend on compiler contraction: binary64 trial
// positions are p + d*u (two roundings) and squared distances dx*dx + dy*dy
// (three roundings); binary32 trial positions are fma(d, u, p) and squared
// distances fma(dx, dx, dy*dy).
#pragma once

#include "hdmc_device.cuh"

namespace hdmc {

template <typename T> struct Vec;
template <> struct Vec<float> { using T2 = float2; };
template <> struct Vec<double> { using T2 = double2; };

// ---- arithmetic of one precision -------------------------------------------
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// trial coordinate p + d*u
__device__ __forceinline__ float trial_coord(float d, float u, float p) { return __fmaf_rn(d, u, p); }
__device__ __forceinline__ double trial_coord(double d, double u, double p) { return __dadd_rn(p, __dmul_rn(d, u)); }

// squared distance compared with sigma^2: overlap iff r^2 < sigma^2
__device__ __forceinline__ bool overlaps(float dx, float dy, float s2) {
    return __fmaf_rn(dx, dx, __fmul_rn(dy, dy)) < s2;
}
__device__ __forceinline__ bool overlaps(double dx, double dy, double s2) {
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < s2;
}

template <typename T> struct Prm;
template <> struct Prm<float> {
    static __device__ __forceinline__ float wx(const Geometry& g) { return g.wxf; }
    static __device__ __forceinline__ float wy(const Geometry& g) { return g.wyf; }
    static __device__ __forceinline__ float d(const Geometry& g) { return g.df; }
    static __device__ __forceinline__ float s2(const Geometry& g) { return g.sig2f; }
    static __device__ __forceinline__ float ds(const SweepDraw& r) { return r.dsf; }
    static __device__ __forceinline__ float prev(float w) { return __uint_as_float(__float_as_uint(w) - 1u); }
    // Direction of a trial move, uniform in the unit disk: two 23-bit
    // symmetric variates per attempt, two attempts per Philox block.
    static __device__ __forceinline__ void direction(const Geometry& g, uint32_t s0, uint32_t s1, uint32_t s2,
                                                     float& u, float& v) {
        uint4 c = make_uint4(s0, s1, s2, 0u);
        for (;;) {
            const uint4 r = philox4x32_10(c, g.key0, g.key1);
            u = sym23(r.x);
            v = sym23(r.y);
            if (__fmaf_rn(u, u, __fmul_rn(v, v)) < 1.0f) return;
            u = sym23(r.z);
            v = sym23(r.w);
            if (__fmaf_rn(u, u, __fmul_rn(v, v)) < 1.0f) return;
            c.w += 1u;
        }
    }
};
template <> struct Prm<double> {
    static __device__ __forceinline__ double wx(const Geometry& g) { return g.wx; }
    static __device__ __forceinline__ double wy(const Geometry& g) { return g.wy; }
    static __device__ __forceinline__ double d(const Geometry& g) { return g.d; }
    static __device__ __forceinline__ double s2(const Geometry& g) { return g.sig2; }
    static __device__ __forceinline__ double ds(const SweepDraw& r) { return r.ds; }
    static __device__ __forceinline__ double prev(double w) {
        return __longlong_as_double(__double_as_longlong(w) - 1ll);
    }
    // Two 52-bit symmetric variates per attempt, one Philox block each.
    static __device__ __forceinline__ void direction(const Geometry& g, uint32_t s0, uint32_t s1, uint32_t s2,
                                                     double& u, double& v) {
        uint4 c = make_uint4(s0, s1, s2, 0u);
        for (;;) {
            const uint4 r = philox4x32_10(c, g.key0, g.key1);
            u = sym52(r.x, r.y);
            v = sym52(r.z, r.w);
            if (__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)) < 1.0) return;
            c.w += 1u;
        }
    }
};

// ---- cell loads / stores -----------------------------------------------------
__device__ __forceinline__ void load_cell(const float2* p, float x[4], float y[4]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    x[0] = a.x; y[0] = a.y; x[1] = a.z; y[1] = a.w;
    x[2] = b.x; y[2] = b.y; x[3] = b.z; y[3] = b.w;
}
__device__ __forceinline__ void load_cell_ro(const float2* p, float x[4], float y[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = a.x; y[0] = a.y; x[1] = a.z; y[1] = a.w;
    x[2] = b.x; y[2] = b.y; x[3] = b.z; y[3] = b.w;
}
__device__ __forceinline__ void store_cell(float2* p, const float x[4], const float y[4]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0], y[0], x[1], y[1]);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[2], y[2], x[3], y[3]);
}
__device__ __forceinline__ void load_cell(const double2* p, double x[4], double y[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double2 a = p[j];
        x[j] = a.x; y[j] = a.y;
    }
}
__device__ __forceinline__ void load_cell_ro(const double2* p, double x[4], double y[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double2 a = __ldg(p + j);
        x[j] = a.x; y[j] = a.y;
    }
}
__device__ __forceinline__ void store_cell(double2* p, const double x[4], const double y[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = make_double2(x[j], y[j]);
}

template <typename T>
__device__ __forceinline__ T pick(const T a[4], int i) {
    return i == 0 ? a[0] : i == 1 ? a[1] : i == 2 ? a[2] : a[3];
}
template <typename T>
__device__ __forceinline__ void put(T a[4], int i, T v) {
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = (i == j) ? v : a[j];
}

__device__ __forceinline__ int wrap(int c, int m) { return c < 0 ? c + m : (c >= m ? c - m : c); }

// ---- sub-sweep: Alg. 1 lines 4-13 / Alg. 2 -----------------------------------
// One thread per active cell of set Q = draw->perm[k]; block 32 x 4 over the
// set's half-resolution grid.  Each thread shuffles its cell, then makes n_M
// trial moves, visiting the shuffled slots cyclically.  A trial is rejected if
// it leaves [0,wx) x [0,wy), else if it overlaps another disk of the cell or a
// disk of the 8 neighbouring cells (translated by their cell offset).  The
// neighbours belong to other sets and are not written by this launch.
template <typename T>
__global__ void __launch_bounds__(128)
k_subsweep(const Geometry g, typename Vec<T>::T2* __restrict__ cells, const SweepDraw* __restrict__ draw, int k,
           unsigned long long* __restrict__ partial) {
    using T2 = typename Vec<T>::T2;
    const int Q = draw->perm[k];
    const uint32_t sweep = draw->sweep;
    const int qx = Q & 1, qy = Q >> 1;
    const int hx = blockIdx.x * 32 + threadIdx.x;
    const int hy = blockIdx.y * 4 + threadIdx.y;
    unsigned int n_tr = 0, n_acc = 0, n_leave = 0;
    if (hx < g.hx && hy < g.hy) {
        const int cx = 2 * hx + qx, cy = 2 * hy + qy;
        T2* own = cells + 4 * ((long long)Q * g.cq + (long long)hy * g.hx + hx);
        T x[4], y[4];
        load_cell(own, x, y);
        const int n = (x[0] >= T(0)) + (x[1] >= T(0)) + (x[2] >= T(0)) + (x[3] >= T(0));
        if (n > 0) {
            const uint32_t cell = (uint32_t)cy * (uint32_t)g.mx + (uint32_t)cx;
            const uint32_t setbits = (uint32_t)Q << 24;
            // Fisher-Yates shuffle of the occupied slots (Alg. 1 line 5)
            if (n >= 2) {
                WordStream s(g.key0, g.key1, sweep, cell, (kDomShuffle << 28) | setbits);
                uint32_t pk = 0x03020100u;   // byte j = old slot now at j
                for (int j = n - 1; j >= 1; --j) {
                    const int kk = (int)s.bounded((uint32_t)(j + 1));
                    const uint32_t aj = (pk >> (8 * j)) & 0xFFu, ak = (pk >> (8 * kk)) & 0xFFu;
                    pk &= ~((0xFFu << (8 * j)) | (0xFFu << (8 * kk)));
                    pk |= (aj << (8 * kk)) | (ak << (8 * j));
                }
                T nx[4], ny[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int src = (pk >> (8 * j)) & 0xFF;
                    nx[j] = pick(x, src);
                    ny[j] = pick(y, src);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) { x[j] = nx[j]; y[j] = ny[j]; }
            }
            // the 8 neighbouring cells, translated into this cell's frame
            T qxs[32], qys[32];
            const T wxs = Prm<T>::wx(g), wys = Prm<T>::wy(g);
            int m = 0;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    const int ncx = wrap(cx + dx, g.mx), ncy = wrap(cy + dy, g.my);
                    T ax[4], ay[4];
                    load_cell_ro(cells + 4 * storage_index(g, ncx, ncy), ax, ay);
                    const T sx = T(dx) * wxs, sy = T(dy) * wys;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        qxs[m + j] = add_rn(ax[j], sx);
                        qys[m + j] = add_rn(ay[j], sy);
                    }
                    m += 4;
                }
            }
            const T d = Prm<T>::d(g), s2 = Prm<T>::s2(g);
            int i = 0;
            for (int t = 0; t < g.nsel; ++t) {
                T u, v;
                Prm<T>::direction(g, sweep, cell, (kDomTrial << 28) | setbits | (uint32_t)t, u, v);
                const T px = pick(x, i), py = pick(y, i);
                const T tx = trial_coord(d, u, px), ty = trial_coord(d, v, py);
                ++n_tr;
                if (tx >= T(0) && tx < wxs && ty >= T(0) && ty < wys) {
                    bool hit = false;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        hit |= (j != i) && overlaps(sub_rn(tx, x[j]), sub_rn(ty, y[j]), s2);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        hit |= overlaps(sub_rn(tx, qxs[j]), sub_rn(ty, qys[j]), s2);
                    if (!hit) {
                        put(x, i, tx);
                        put(y, i, ty);
                        ++n_acc;
                    }
                } else {
                    ++n_leave;
                }
                i = (i + 1 == n) ? 0 : i + 1;
            }
            store_cell(own, x, y);
        }
    }
    // per-block counters: partial[4b + {trials, accepted, left, overlap}]
    __shared__ unsigned int red[4][3];
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
        const unsigned tr = red[0][0] + red[1][0] + red[2][0] + red[3][0];
        const unsigned ac = red[0][1] + red[1][1] + red[2][1] + red[3][1];
        const unsigned lv = red[0][2] + red[1][2] + red[2][2] + red[3][2];
        unsigned long long* p = partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
        p[0] += tr;
        p[1] += ac;
        p[2] += lv;
        p[3] += tr - ac - lv;
    }
}

// ---- cell shift: Alg. 4 ---------------------------------------------------------
// One thread per new cell (storage order).  New cell c = the disks of old c
// that stay inside c after the translation by -f*ds (old slot order), then
// the disks of old c+f that leave c+f, re-expressed in c's frame (+f*w).  The
// ownership test is the same expression in the two threads that see a disk,
// so every disk lands in exactly one cell (Sec. 3.2).  A re-expressed value
// that rounds onto the upper edge is clamped to the largest value below it.
template <typename T>
__global__ void __launch_bounds__(256)
k_shift(const Geometry g, const typename Vec<T>::T2* __restrict__ src, typename Vec<T>::T2* __restrict__ dst,
        const SweepDraw* __restrict__ draw, DevState* __restrict__ st) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int fdir = draw->fdir;
    const int ax = fdir >> 1;
    const int sgn = (fdir & 1) ? -1 : 1;
    const T w = ax ? Prm<T>::wy(g) : Prm<T>::wx(g);
    const T sd = T(sgn) * Prm<T>::ds(*draw);
    const T sw = T(sgn) * w;
    if (idx == 0) st->origin[ax] += (double)sd;
    if (idx >= g.C) return;
    const int q = (int)(idx / g.cq);
    const long long r = idx - (long long)q * g.cq;
    const int hy = (int)(r / g.hx);
    const int hx = (int)(r - (long long)hy * g.hx);
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    const int ncx = ax ? cx : wrap(cx + sgn, g.mx);
    const int ncy = ax ? wrap(cy + sgn, g.my) : cy;
    T ox[4], oy[4], bx[4], by[4];
    load_cell_ro(src + 4 * idx, ox, oy);
    load_cell_ro(src + 4 * storage_index(g, ncx, ncy), bx, by);
    T rx[4], ry[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { rx[j] = T(kEmpty); ry[j] = T(kEmpty); }
    int kept = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (ox[j] >= T(0)) {
            const T dp = sub_rn(ax ? oy[j] : ox[j], sd);
            if (dp >= T(0) && dp < w) {
                const T vx = ax ? ox[j] : dp, vy = ax ? dp : oy[j];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    rx[s] = (kept == s) ? vx : rx[s];
                    ry[s] = (kept == s) ? vy : ry[s];
                }
                ++kept;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (bx[j] >= T(0)) {
            const T dp = sub_rn(ax ? by[j] : bx[j], sd);
            if (!(dp >= T(0) && dp < w)) {
                T v = add_rn(dp, sw);
                v = (v >= w) ? Prm<T>::prev(w) : v;
                v = (v < T(0)) ? T(0) : v;
                const T vx = ax ? bx[j] : v, vy = ax ? v : by[j];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    rx[s] = (kept == s) ? vx : rx[s];
                    ry[s] = (kept == s) ? vy : ry[s];
                }
                ++kept;
            }
        }
    }
    if (kept > 4) atomicOr(&st->error, 1u);
    store_cell(dst + 4 * idx, rx, ry);
}

// ---- contact histogram: Sec. 4 ------------------------------------------------------
// Ordered pairs (i, j != i) at distance r in [sigma, sigma + 200 dr), bin
// floor((r - sigma)/dr), distances in binary64 from cell-local coordinates
// over the 5x5 neighbourhood (w >= sigma, so two rings reach past 1.02 sigma).
// Grid-stride over cells; per-block shared histogram, one atomic per bin.
template <typename T>
__global__ void __launch_bounds__(256)
k_hist(const Geometry g, const typename Vec<T>::T2* __restrict__ cells, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int sh[kHistBins];
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const double wxd = (double)Prm<T>::wx(g), wyd = (double)Prm<T>::wy(g);
    const double sigma = g.sigma, dr = kHistDr * g.sigma;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.C;
         idx += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(idx / g.cq);
        const long long r = idx - (long long)q * g.cq;
        const int hy = (int)(r / g.hx);
        const int hx = (int)(r - (long long)hy * g.hx);
        const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
        T px[4], py[4];
        load_cell_ro(cells + 4 * idx, px, py);
        if (!(px[0] >= T(0))) continue;
        for (int dy = -2; dy <= 2; ++dy) {
            for (int dx = -2; dx <= 2; ++dx) {
                const int ncx = wrap(cx + dx, g.mx), ncy = wrap(cy + dy, g.my);
                T qx[4], qy[4];
                load_cell_ro(cells + 4 * storage_index(g, ncx, ncy), qx, qy);
                const double sx = (double)dx * wxd, sy = (double)dy * wyd;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!(qx[j] >= T(0))) continue;
                    const double ex = __dadd_rn((double)qx[j], sx), ey = __dadd_rn((double)qy[j], sy);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!(px[i] >= T(0))) continue;
                        if (dx == 0 && dy == 0 && i == j) continue;
                        const double ddx = __dsub_rn((double)px[i], ex), ddy = __dsub_rn((double)py[i], ey);
                        const double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)));
                        const double t = __ddiv_rn(__dsub_rn(rr, sigma), dr);
                        if (t >= 0.0 && t < (double)kHistBins) atomicAdd(&sh[(int)t], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// ---- launchers ---------------------------------------------------------------------
template <typename T>
void launch_subsweep_t(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k) {
    k_subsweep<T><<<subsweep_grid(c.g), dim3(32, 4), 0, c.stream>>>(
        c.g, reinterpret_cast<typename Vec<T>::T2*>(cells), draw, k, c.partial);
}

template <typename T>
void launch_shift_t(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw) {
    const long long blocks = (c.g.C + 255) / 256;
    k_shift<T><<<(unsigned)blocks, 256, 0, c.stream>>>(
        c.g, reinterpret_cast<const typename Vec<T>::T2*>(src), reinterpret_cast<typename Vec<T>::T2*>(dst), draw,
        c.st);
}

template <typename T>
void launch_hist_t(const LaunchCtx& c, const void* cells) {
    long long blocks = (c.g.C + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_hist<T><<<(unsigned)blocks, 256, 0, c.stream>>>(c.g, reinterpret_cast<const typename Vec<T>::T2*>(cells),
                                                      c.hist);
}

}  // namespace hdmc
