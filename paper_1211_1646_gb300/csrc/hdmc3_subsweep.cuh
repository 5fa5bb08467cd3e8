// hdmc3_subsweep.cuh -- the three-dimensional sub-sweep (Alg. 1 and Alg. 2
// with eight checkerboard sets): one thread per active cell.  Before its
// trials a thread gathers, into shared memory, the spheres of its 26
// neighbour cells within reach of the box that holds all its trial positions;
// no other sphere can overlap a trial position, so the decisions are those of
// testing the whole neighbourhood, and every test keeps the arithmetic of the
// serial form.
#pragma once

#include "hdmc3_device.cuh"

namespace hdmc {

// Is (hi:lo, ...) an attempt inside the unit ball?  The definition is the
// binary64 test (u0*u0 + u1*u1) + u2*u2 < 1 on the three sym52 variates.  A
// binary32 estimate from the high words (each within 6.1e-8 of its variate,
// so the estimate of the sum within 1e-6) decides whenever it lies farther
// than 2^-16 from 1; the rest are decided in binary64.
__device__ __forceinline__ bool inside_ball(const uint32_t (&w)[6]) {
    const float a = (float)(int32_t)(w[0] ^ 0x80000000u) * 0x1p-31f;
    const float b = (float)(int32_t)(w[2] ^ 0x80000000u) * 0x1p-31f;
    const float c = (float)(int32_t)(w[4] ^ 0x80000000u) * 0x1p-31f;
    const float s = a * a + b * b + c * c;
    if (s < 1.0f - 0x1p-16f) return true;
    if (s > 1.0f + 0x1p-16f) return false;
    const double u0 = sym52(w[0], w[1]), u1 = sym52(w[2], w[3]), u2 = sym52(w[4], w[5]);
    return (u0 * u0 + u1 * u1) + u2 * u2 < 1.0;
}

// Trial directions of one cell update, uniform in the unit ball by
// rejection from (-1,1)^3.
//   binary64: consecutive words of the trial stream, six per attempt,
//             three sym52 variates;
//   binary32: each Philox block of the trial stream cut into six 21-bit
//             fields, two attempts of three sym21 variates per block, kept
//             when fma(u, u, fma(v, v, s*s)) < 1.
template <typename T> struct TrialDir;
template <> struct TrialDir<double> {
    WordStream ws;
    __device__ TrialDir(const G3& g, uint32_t sweep, uint32_t c, uint32_t dom) : ws(g.key0, g.key1, sweep, c, dom) {}
    // The next `want` kept directions into column threadIdx.x of u, with the
    // lanes that still need one drawing their attempts together (from a
    // common start they stay at the same word of their streams, so the
    // Philox blocks are computed converged).
    __device__ __forceinline__ void fill(int want, double (*u)[3][kSubB3]) {
        for (int have = 0; have < want;) {
            uint32_t wd[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) wd[q] = ws.next();
            if (inside_ball(wd)) {
                u[have][0][threadIdx.x] = sym52(wd[0], wd[1]);
                u[have][1][threadIdx.x] = sym52(wd[2], wd[3]);
                u[have][2][threadIdx.x] = sym52(wd[4], wd[5]);
                ++have;
            }
        }
    }
};
template <> struct TrialDir<float> {
    uint32_t k0, k1, sweep, c, dom, block;
    uint32_t f[6];
    int triple;
    __device__ TrialDir(const G3& g, uint32_t sweep_, uint32_t c_, uint32_t dom_)
        : k0(g.key0), k1(g.key1), sweep(sweep_), c(c_), dom(dom_), block(0), triple(2) {}
    // The next `want` kept directions (attempts in stream order: the field
    // triples (0,1,2) and (3,4,5) of block 0, then of block 1, ...) into
    // column threadIdx.x of u.  Lanes that still need a direction compute
    // their next Philox block together, so the generator runs with the warp
    // converged, not once for every lane that happens to need a block in a
    // given trial.
    __device__ __forceinline__ void fill(int want, float (*u)[3][kSubB3]) {
        int have = 0;
        for (;;) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (triple == a && have < want) {
                    const float u0 = sym21(f[3 * a]), u1 = sym21(f[3 * a + 1]), u2 = sym21(f[3 * a + 2]);
                    ++triple;
                    if (fmaf(u0, u0, fmaf(u1, u1, u2 * u2)) < 1.0f) {
                        u[have][0][threadIdx.x] = u0;
                        u[have][1][threadIdx.x] = u1;
                        u[have][2][threadIdx.x] = u2;
                        ++have;
                    }
                }
            }
            if (have >= want) break;
            fields21(philox4x32_10(make_uint4(sweep, c, dom, block), k0, k1), f);
            ++block;
            triple = 0;
        }
    }
};

// Trial directions drawn ahead per thread (shared memory).
constexpr int kDir3 = 4;
template <typename T> struct DirBuf { T u[kDir3][3][kSubB3]; };

// Pair test on binary32 copies of the coordinates: 1 overlap, 0 none, 2 too
// close to contact for binary32 to decide (binary64 only; the copies are
// within 3e-7 of the binary64 values, so r^2 is within 1e-5 of the binary64
// one, well inside the 2^-14 sigma^2 band).  In binary32 mode the copies are
// the coordinates and this is the method's own test.
template <typename T>
__device__ __forceinline__ int quick_hit(const G3& g, float dx, float dy, float dz);
template <>
__device__ __forceinline__ int quick_hit<float>(const G3& g, float dx, float dy, float dz) {
    return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, -g.sig2f))) < 0.0f;
}
template <>
__device__ __forceinline__ int quick_hit<double>(const G3& g, float dx, float dy, float dz) {
    const float r2 = dx * dx + dy * dy + dz * dz;
    return r2 < g.band_lo ? 1 : (r2 > g.band_hi ? 0 : 2);
}

// Exact test of the trial position against every sphere of the neighbour
// cell with storage index sn (its offset from the cell (cx,cy,cz) is
// recovered from the grid: m >= 4 makes it unique).
template <typename T>
__device__ bool cell_hit_exact(const G3& g, const T* cells, unsigned sn, int cx, int cy, int cz, T px, T py, T pz) {
    using A = Ar3<T>;
    const unsigned Q = sn / g.cq, r0 = sn % g.cq;
    const int ix = (int)(r0 % (unsigned)g.h[0]);
    const unsigned r1 = r0 / (unsigned)g.h[0];
    const int iy = (int)(r1 % (unsigned)g.h[1]), iz = (int)(r1 / (unsigned)g.h[1]);
    int dd[3] = {2 * ix + (int)(Q & 1) - cx, 2 * iy + (int)((Q >> 1) & 1) - cy, 2 * iz + (int)(Q >> 2) - cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) dd[a] = dd[a] > 1 ? dd[a] - g.m[a] : (dd[a] < -1 ? dd[a] + g.m[a] : dd[a]);
    const T sx = (T)dd[0] * A::w(g, 0), sy = (T)dd[1] * A::w(g, 1), sz = (T)dd[2] * A::w(g, 2);
    bool hit = false;
    for (int j = 0; j < kSlots3; ++j) {
        const T* q = slot3(cells, g, sn, j);
        if (q[0] == (T)kEmpty) break;
        hit |= A::hit(g, px - (q[0] + sx), py - (q[4] + sy), pz - (q[8] + sz));
    }
    return hit;
}

// Does the trial position hit a sphere of the 26 neighbour cells?  Reads
// global memory (used when a cell has more than kCand3 gathered spheres).
template <typename T>
__device__ bool neighbour_hit_global(const G3& g, const T* cells, int cx, int cy, int cz, T px, T py, T pz) {
    using A = Ar3<T>;
    bool hit = false;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const unsigned sn = sidx3(g, wrap3(cx + dx, g.m[0]), wrap3(cy + dy, g.m[1]), wrap3(cz + dz, g.m[2]));
                const T sx = (T)dx * A::w(g, 0), sy = (T)dy * A::w(g, 1), sz = (T)dz * A::w(g, 2);
                for (int j = 0; j < kSlots3; ++j) {
                    const T* q = slot3(cells, g, sn, j);
                    if (q[0] == (T)kEmpty) break;
                    const T ex = q[0] + sx, ey = q[4] + sy, ez = q[8] + sz;
                    hit |= A::hit(g, px - ex, py - ey, pz - ez);
                }
            }
    return hit;
}

// Per-thread candidate lists in shared memory, column t for thread t:
// binary32 keeps the three coordinates (12 bytes a candidate); binary64 adds
// the neighbour cell's storage index for the exact test near contact.
template <typename T> struct Cand;
template <> struct Cand<float> {
    float x[kCand3][kSubB3], y[kCand3][kSubB3], z[kCand3][kSubB3];
    __device__ __forceinline__ void put(int q, float a, float b, float c, unsigned) {
        x[q][threadIdx.x] = a;
        y[q][threadIdx.x] = b;
        z[q][threadIdx.x] = c;
    }
    __device__ __forceinline__ float4 get(int q) const {
        return make_float4(x[q][threadIdx.x], y[q][threadIdx.x], z[q][threadIdx.x], 0.0f);
    }
};
template <> struct Cand<double> {
    float4 v[kCand3][kSubB3];
    __device__ __forceinline__ void put(int q, float a, float b, float c, unsigned sn) {
        v[q][threadIdx.x] = make_float4(a, b, c, __uint_as_float(sn));
    }
    __device__ __forceinline__ float4 get(int q) const { return v[q][threadIdx.x]; }
};

// Gather the occupied slots of one half of a neighbour cell (offset
// dx,dy,dz, storage index sn) that lie within reach of the box [lo, hi] that
// holds every trial position of this cell update: their binary32 image
// coordinates (and sn in binary64) go to the thread's candidate list.
template <typename T>
__device__ __forceinline__ void gather_half(const G3& g, const T (&qx)[4], const T (&qy)[4], const T (&qz)[4],
                                            int dx, int dy, int dz, unsigned sn, const float (&lo)[3],
                                            const float (&hi)[3], Cand<T>& cand, int& nc) {
    const float sx = (float)dx * g.wf[0], sy = (float)dy * g.wf[1], sz = (float)dz * g.wf[2];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if constexpr (sizeof(T) == 4) {
            // without branches: an empty slot's sentinel lies far outside the
            // reach of any box, and a candidate that is not kept is
            // overwritten by the next one (3 % faster than the branches)
            const float ex = qx[j] + sx, ey = qy[j] + sy, ez = qz[j] + sz;
            const float gx = fmaxf(fmaxf(lo[0] - ex, ex - hi[0]), 0.0f);
            const float gy = fmaxf(fmaxf(lo[1] - ey, ey - hi[1]), 0.0f);
            const float gz = fmaxf(fmaxf(lo[2] - ez, ez - hi[2]), 0.0f);
            const bool keep = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < g.keep2f;
            if (nc < kCand3) cand.put(nc, ex, ey, ez, sn);
            nc += keep;
        } else if (qx[j] != (T)kEmpty) {   // binary64: convert only occupied slots
            const float ex = (float)qx[j] + sx, ey = (float)qy[j] + sy, ez = (float)qz[j] + sz;
            const float gx = fmaxf(fmaxf(lo[0] - ex, ex - hi[0]), 0.0f);
            const float gy = fmaxf(fmaxf(lo[1] - ey, ey - hi[1]), 0.0f);
            const float gz = fmaxf(fmaxf(lo[2] - ez, ez - hi[2]), 0.0f);
            if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < g.keep2f) {
                if (nc < kCand3) cand.put(nc, ex, ey, ez, sn);
                ++nc;
            }
        }
    }
}

// Both halves of a neighbour cell whose primary half is already loaded.
template <typename T>
__device__ __forceinline__ void gather_cell(const G3& g, const T* cells, const T (&qx)[4], const T (&qy)[4],
                                            const T (&qz)[4], int dx, int dy, int dz, unsigned sn,
                                            const float (&lo)[3], const float (&hi)[3], Cand<T>& cand, int& nc) {
    gather_half(g, qx, qy, qz, dx, dy, dz, sn, lo, hi, cand, nc);
    if (qx[3] != (T)kEmpty) {
        const T* p = cells + secondary3(g, sn);
        T rx[4], ry[4], rz[4];
        ld4(p, rx);
        ld4(p + 4, ry);
        ld4(p + 8, rz);
        gather_half(g, rx, ry, rz, dx, dy, dz, sn, lo, hi, cand, nc);
    }
}

// One sub-sweep: every cell of set Q = table[jd].perm[k] (Alg. 1, Alg. 2).
// binary32: the neighbour cells of one x-row are loaded together (256-bit
// loads) before they are scanned; binary64: one cell at a time.
template <typename T>
__device__ __forceinline__ void sub3_cells(const G3& g, T* __restrict__ cells, const Draw3* __restrict__ table, int jd,
                                           int k, Dev3* st) {
    using A = Ar3<T>;
    __shared__ Cand<T> cand;
    __shared__ DirBuf<T> dirs;
    const Draw3& dr = table[jd];
    const int Q = dr.perm[k];
    const unsigned s = blockIdx.x * kSubB3 + threadIdx.x;
    uint32_t n_tr = 0, n_ac = 0, n_lf = 0, n_ov = 0;
    if (s < g.cq) {
        const int ix = (int)(s % (unsigned)g.h[0]);
        const unsigned r = s / (unsigned)g.h[0];
        const int iy = (int)(r % (unsigned)g.h[1]);
        const int iz = (int)(r / (unsigned)g.h[1]);
        const int cx = 2 * ix + (Q & 1), cy = 2 * iy + ((Q >> 1) & 1), cz = 2 * iz + (Q >> 2);
        const unsigned sown = (unsigned)Q * g.cq + s;
        T x[8], y[8], z[8];
        ld_cell3(cells, g, sown, x, y, z);
        int n = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) n += x[j] != (T)kEmpty;
        if (n > 0) {
            const uint32_t c = ((uint32_t)cz * (uint32_t)g.m[1] + (uint32_t)cy) * (uint32_t)g.m[0] + (uint32_t)cx;
            const uint32_t setbits = (uint32_t)Q << 24;
            if (n >= 2 && !(g.flags & kNoParticleShuffle)) {
                WordStream S(g.key0, g.key1, dr.sweep, c, (kDomShuffle << 28) | setbits);
                shuffle3(x, y, z, n, S.bounded(factorial8(n)));
            }
            // Every trial position lies in the box [lo, hi]: a sphere makes at
            // most K = ceil(n_M / n) trials, each moving it by less than d per
            // axis from where the previous accepted one left it, and positions
            // outside [0, w) are rejected before any overlap test.
            float lo[3], hi[3];
            {
                const int K = (g.nsel + n - 1) / n;
                const float reach = (float)K * g.df * (1.0f + 1.0e-5f) + 1.0e-6f;
                float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < n) {
                        const float v[3] = {(float)x[j], (float)y[j], (float)z[j]};
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            mn[a] = fminf(mn[a], v[a]);
                            mx[a] = fmaxf(mx[a], v[a]);
                        }
                    }
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[a] = fmaxf(0.0f, mn[a] - reach);
                    hi[a] = fminf(g.wf[a], mx[a] + reach);
                }
            }
            int nc = 0;
#pragma unroll 1
            for (int row = 0; row < 9; ++row) {
                const int dz = row / 3 - 1, dy = row % 3 - 1;
                const int ny = wrap3(cy + dy, g.m[1]), nz = wrap3(cz + dz, g.m[2]);
                if (sizeof(T) == 4) {
                    T ax[3][4], ay[3][4], az[3][4];
                    unsigned sn[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        sn[e] = sidx3(g, wrap3(cx + e - 1, g.m[0]), ny, nz);
                        const T* p = cells + primary3(sn[e]);
                        ld4(p, ax[e]);
                        ld4(p + 4, ay[e]);
                        ld4(p + 8, az[e]);
                    }
#pragma unroll
                    for (int e = 0; e < 3; ++e)
                        if (e != 1 || row != 4)
                            gather_cell(g, cells, ax[e], ay[e], az[e], e - 1, dy, dz, sn[e], lo, hi, cand, nc);
                } else {
#pragma unroll 1
                    for (int e = 0; e < 3; ++e) {
                        if (e == 1 && row == 4) continue;
                        const unsigned sn = sidx3(g, wrap3(cx + e - 1, g.m[0]), ny, nz);
                        const T* p = cells + primary3(sn);
                        T ax[4], ay[4], az[4];
                        ld4(p, ax);
                        ld4(p + 4, ay);
                        ld4(p + 8, az);
                        gather_cell(g, cells, ax, ay, az, e - 1, dy, dz, sn, lo, hi, cand, nc);
                    }
                }
            }
            const bool spill = nc > kCand3;
            float fx[8], fy[8], fz[8];   // binary32 copies of the own coordinates
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                fx[j] = (float)x[j];
                fy[j] = (float)y[j];
                fz[j] = (float)z[j];
            }
            const T w0 = A::w(g, 0), w1 = A::w(g, 1), w2 = A::w(g, 2);
            TrialDir<T> TD(g, dr.sweep, c, (kDomTrial << 28) | setbits);
            int i = 0;
            for (int t = 0; t < g.nsel; ++t) {
                T u0, u1, u2;
                {   // drawn ahead, kDir3 at a time
                    const int tt = t % kDir3;
                    if (tt == 0) TD.fill(min(kDir3, g.nsel - t), dirs.u);
                    u0 = dirs.u[tt][0][threadIdx.x];
                    u1 = dirs.u[tt][1][threadIdx.x];
                    u2 = dirs.u[tt][2][threadIdx.x];
                }
                const T px = A::trial(g, pick8(x, i), u0);
                const T py = A::trial(g, pick8(y, i), u1);
                const T pz = A::trial(g, pick8(z, i), u2);
                ++n_tr;
                if (!(px >= (T)0 && px < w0 && py >= (T)0 && py < w1 && pz >= (T)0 && pz < w2)) {
                    ++n_lf;
                } else {
                    const float pfx = (float)px, pfy = (float)py, pfz = (float)pz;
                    bool hit = false;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j < n && j != i) {
                            int h = quick_hit<T>(g, pfx - fx[j], pfy - fy[j], pfz - fz[j]);
                            if (h == 2) h = A::hit(g, px - x[j], py - y[j], pz - z[j]);
                            hit |= h != 0;
                        }
                    if (!spill) {
                        int q = 0;
                        for (; q + 1 < nc && !hit; q += 2) {
                            const float4 e0 = cand.get(q), e1 = cand.get(q + 1);
                            int h0 = quick_hit<T>(g, pfx - e0.x, pfy - e0.y, pfz - e0.z);
                            int h1 = quick_hit<T>(g, pfx - e1.x, pfy - e1.y, pfz - e1.z);
                            if (h0 == 2) h0 = cell_hit_exact(g, cells, __float_as_uint(e0.w), cx, cy, cz, px, py, pz);
                            if (h1 == 2) h1 = cell_hit_exact(g, cells, __float_as_uint(e1.w), cx, cy, cz, px, py, pz);
                            hit = (h0 | h1) != 0;
                        }
                        if (q < nc && !hit) {
                            const float4 e = cand.get(q);
                            int h = quick_hit<T>(g, pfx - e.x, pfy - e.y, pfz - e.z);
                            if (h == 2) h = cell_hit_exact(g, cells, __float_as_uint(e.w), cx, cy, cz, px, py, pz);
                            hit = h != 0;
                        }
                    } else if (!hit) {
                        hit = neighbour_hit_global(g, cells, cx, cy, cz, px, py, pz);
                    }
                    if (hit) {
                        ++n_ov;
                    } else {
                        put8(x, i, px);
                        put8(y, i, py);
                        put8(z, i, pz);
                        put8(fx, i, pfx);
                        put8(fy, i, pfy);
                        put8(fz, i, pfz);
                        ++n_ac;
                    }
                }
                i = i + 1 == n ? 0 : i + 1;
            }
            st_cell3(cells, g, sown, x, y, z, n > 4);
        }
    }
    const unsigned a = __reduce_add_sync(0xFFFFFFFFu, n_tr), b = __reduce_add_sync(0xFFFFFFFFu, n_ac);
    const unsigned cc = __reduce_add_sync(0xFFFFFFFFu, n_lf), d = __reduce_add_sync(0xFFFFFFFFu, n_ov);
    if ((threadIdx.x & 31) == 0 && a) {
        atomicAdd(&st->ctr[0], (unsigned long long)a);
        atomicAdd(&st->ctr[1], (unsigned long long)b);
        atomicAdd(&st->ctr[2], (unsigned long long)cc);
        atomicAdd(&st->ctr[3], (unsigned long long)d);
    }
}

template <typename T>
__global__ void __launch_bounds__(kSubB3) k_sub3(G3 g, T* __restrict__ cells, const Draw3* __restrict__ table, int jd,
                                                 int k, Dev3* st) {
    sub3_cells<T>(g, cells, table, jd, k, st);
}
// binary32: eight blocks per SM (128 registers; ten blocks at 96 registers
// spill and measured slower, 46.8 against 41.5 us)
template <>
__global__ void __launch_bounds__(kSubB3, 8) k_sub3<float>(G3 g, float* __restrict__ cells,
                                                            const Draw3* __restrict__ table, int jd, int k, Dev3* st) {
    sub3_cells<float>(g, cells, table, jd, k, st);
}

}  // namespace hdmc
