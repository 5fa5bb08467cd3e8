// hdmc3.cu -- the method in three dimensions: hard spheres in cubic cells,
// eight checkerboard sets (the paper describes the 3-d case in words:
// Sec. 2.1 and 2.2 give eight sets and eight sub-sweeps per sweep, Sec. 6
// discusses hard spheres).  Kernels and host entry points of the hdmc3_*
// part of the C ABI.
//
// Layout and shared helpers: hdmc3_device.cuh; the sub-sweep kernel:
// hdmc3_subsweep.cuh.
//
// Random streams (Philox4x32-10 keyed by the seed), with c the canonical cell
// number (cz*my + cy)*mx + cx:
//   sweep draws of sweep s:          (s, 0xFFFFFFFF, 2<<28): Fisher-Yates
//                                    order of the 8 sets, direction f in 0..5,
//                                    distance unif53 * w/2
//   explicit shift k:                (k, 0xFFFFFFFF, 4<<28): f, distance
//   shuffle of cell c, sweep s, Q:   (s, c, (0<<28)|(Q<<24)): k in [0, n!)
//   trials of that update:           (s, c, (1<<28)|(Q<<24)): directions
//                                    kept inside the unit ball (binary64:
//                                    six words per attempt, three sym52;
//                                    binary32: two attempts of three 21-bit
//                                    fields per block)
//   start jitter of sphere p:        (p, 0xFFFFFFFE, 3<<28)

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hdmc.h"
#include "hdmc3_subsweep.cuh"

namespace hdmc {

// Host helpers of the two-dimensional entry points (hdmc_host.cu).
int cuda_code(cudaError_t e);
int error_code(unsigned int device_error);
void bin_axis(double x, double w, int m, int& cell, double& loc);
double poly_intercept(const std::vector<double>& t, const std::vector<double>& y, int deg);
void squared_edges(double sigma, double* E);

// Sweep or shift draws for `count` consecutive indices starting at `first`.
__global__ void k_draws3(G3 g, Draw3* table, uint32_t first, int count, int sweep_mode) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t index = first + (uint32_t)i;
    WordStream s(g.key0, g.key1, index, 0xFFFFFFFFu, (sweep_mode ? kDomSweep : kDomShift) << 28);
    int p[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    if (sweep_mode) {
#pragma unroll
        for (int j = 7; j >= 1; --j) {
            const int k = (int)s.bounded((uint32_t)(j + 1));
            const int t = p[j];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q == k) {
                    p[j] = p[q];
                    p[q] = t;
                }
        }
    }
    Draw3 r;
    const bool fixed = (g.flags & kNoSetShuffle) != 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) r.perm[q] = (uint8_t)(fixed ? q : p[q]);
    r.fdir = (int32_t)s.bounded(6u);
    const uint32_t hi = s.next();
    const uint32_t lo = s.next();
    const int ax = r.fdir >> 1;
    const double w = ax == 0 ? g.w[0] : (ax == 1 ? g.w[1] : g.w[2]);
    r.ds = unif53(hi, lo) * (0.5 * w);
    r.sweep = index;
    table[i] = r;
}

// Cell shift (Alg. 4) along one of three axes: new cell c keeps the spheres
// of old c that stay inside it (slot order), then takes those of old c+f
// that leave c+f, re-expressed in c's frame and clamped into [0, w).  Both
// old cells are read with 256-bit loads and the new cell is put together in
// registers.
template <typename T>
__device__ __forceinline__ T sel3(int ax, T a, T b, T c) {
    return ax == 0 ? a : (ax == 1 ? b : c);
}

template <typename T>
__global__ void __launch_bounds__(kShiftB3) k_shift3(G3 g, const T* __restrict__ src, T* __restrict__ dst,
                                                     const Draw3* __restrict__ table, int jd, Dev3* st) {
    const unsigned s = blockIdx.x * kShiftB3 + threadIdx.x;
    if (s >= g.C) return;
    const Draw3& dr = table[jd];
    const int ax = dr.fdir >> 1;
    const int sgn = (dr.fdir & 1) ? -1 : 1;
    const unsigned Q = s / g.cq, r0 = s % g.cq;
    const int ix = (int)(r0 % (unsigned)g.h[0]);
    const unsigned r1 = r0 / (unsigned)g.h[0];
    const int iy = (int)(r1 % (unsigned)g.h[1]), iz = (int)(r1 / (unsigned)g.h[1]);
    int nx = 2 * ix + (int)(Q & 1), ny = 2 * iy + (int)((Q >> 1) & 1), nz = 2 * iz + (int)(Q >> 2);
    if (ax == 0) nx = wrap3(nx + sgn, g.m[0]);
    else if (ax == 1) ny = wrap3(ny + sgn, g.m[1]);
    else nz = wrap3(nz + sgn, g.m[2]);
    T ox[8], oy[8], oz[8], bx[8], by[8], bz[8];
    ld_cell3(src, g, s, ox, oy, oz);
    ld_cell3(src, g, sidx3(g, nx, ny, nz), bx, by, bz);
    T w, sd, sw, wprev;
    if (sizeof(T) == 8) {
        w = (T)g.w[ax];
        sd = (T)((double)sgn * dr.ds);
        sw = (T)((double)sgn * g.w[ax]);
        wprev = (T)g.wprev[ax];
    } else {
        w = (T)g.wf[ax];
        sd = (T)((float)sgn * (float)dr.ds);
        sw = (T)((float)sgn * g.wf[ax]);
        wprev = (T)g.wprevf[ax];
    }
    T rx[8], ry[8], rz[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) rx[j] = ry[j] = rz[j] = (T)kEmpty;
    int k = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const T dp = sel3(ax, ox[j], oy[j], oz[j]) - sd;
        if (ox[j] != (T)kEmpty && dp >= (T)0 && dp < w) {
            put8(rx, k, ax == 0 ? dp : ox[j]);
            put8(ry, k, ax == 1 ? dp : oy[j]);
            put8(rz, k, ax == 2 ? dp : oz[j]);
            ++k;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const T dp = sel3(ax, bx[j], by[j], bz[j]) - sd;
        if (bx[j] != (T)kEmpty && !(dp >= (T)0 && dp < w)) {
            T v = dp + sw;
            if (v >= w) v = wprev;
            if (v < (T)0) v = (T)0;
            put8(rx, k, ax == 0 ? v : bx[j]);
            put8(ry, k, ax == 1 ? v : by[j]);
            put8(rz, k, ax == 2 ? v : bz[j]);
            ++k;
        }
    }
    if (k > kSlots3) atomicOr(&st->error, kErrOverflow);
    st_cell3(dst, g, s, rx, ry, rz, k >= 4);
    if (s == 0) st->origin[ax] += (double)sd;
}

// Contact histogram: every sphere against the spheres of its 5x5x5 cell
// neighbourhood; a binary32 estimate of r^2 with a wide margin skips pairs
// far outside [sigma^2, (sigma + 200 dr)^2), the rest are decided in binary64
// on r^2 = (dx*dx + dy*dy) + dz*dz against the squared bin edges.  One thread
// per cell: its spheres stay in registers while the neighbour cells are read
// once each.  A cell two steps away along an axis is read only if one of the
// cell's spheres is within reach of it along that axis (its face is closer
// than sigma + 200 dr, with a relative margin of 1e-5); with w close to sigma
// that is rare, so most cells read 27 neighbours instead of 125.  Binary64
// arithmetic is used only for the pairs the binary32 estimate cannot exclude.
__device__ __forceinline__ void hist_bin(double r2, const double* __restrict__ edges2, unsigned int* sh) {
    if (!(r2 >= edges2[0]) || !(r2 < edges2[kHistBins])) return;
    int lo = 0, hi = kHistBins;   // largest b with edges2[b] <= r2
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (r2 >= edges2[mid]) lo = mid;
        else hi = mid;
    }
    atomicAdd(&sh[lo], 1u);
}

// The binary64 decision for one pair that the binary32 estimate could not
// exclude: r^2 = (e0*e0 + e1*e1) + e2*e2 with e = p - (q + d w), as the serial
// form computes it.  Kept out of line so that the compiler cannot evaluate it
// speculatively for every pair (binary64 is slow on GB300).
template <typename T>
__device__ __noinline__ void hist_pair_exact(T ax, T ay, T az, T qx, T qy, T qz, int dx, int dy, int dz, double w0,
                                             double w1, double w2, const double* __restrict__ edges2,
                                             unsigned int* sh) {
    const double e0 = (double)ax - ((double)qx + (double)dx * w0);
    const double e1 = (double)ay - ((double)qy + (double)dy * w1);
    const double e2 = (double)az - ((double)qz + (double)dz * w2);
    hist_bin((e0 * e0 + e1 * e1) + e2 * e2, edges2, sh);
}

// Binary32 bounds that decide a pair's bin without binary64 arithmetic.  The
// binary32 estimate r2f (coordinates rounded to binary32, differences and
// squares in binary32) lies within kBinMargin sigma^2 of the binary64 r^2
// the bins are defined on: per axis the estimate's difference is off by at
// most 7 units of 2^-24 sigma-scaled (|q + d w| <= 3.5 sigma, |p - q - d w|
// <= 1.03 sigma in the histogram's range, the two roundings of a binary64
// coordinate), hence r^2 by at most 2 sqrt(3) 1.03 (4.2e-7) + 3 (1.04) 2^-24
// < 1.7e-6 sigma^2; the margin is 4e-6 sigma^2.  B[2b], B[2b+1] (b < 200):
// r2f in [B[2b], B[2b+1]) puts the pair in bin b for certain; B[400]: r2f
// below it is below every bin; B[401]: r2f at or above it is above them.
constexpr double kBinMargin = 4.0e-6;
static float float_up(double x) {
    float f = (float)x;
    return (double)f < x ? std::nextafter(f, HUGE_VALF) : f;
}
static float float_down(double x) {
    float f = (float)x;
    return (double)f > x ? std::nextafter(f, -HUGE_VALF) : f;
}
static void certified_bins(double sigma, const double* E, float* B) {
    const double m = kBinMargin * sigma * sigma;
    for (int b = 0; b < kHistBins; ++b) {
        B[2 * b] = float_up(E[b] + m);
        B[2 * b + 1] = float_down(E[b + 1] - m);
    }
    B[2 * kHistBins] = float_down(E[0] - m);
    B[2 * kHistBins + 1] = float_up(E[kHistBins] + m);
}

template <typename T>
__global__ void __launch_bounds__(kHistB3, 4) k_hist3(G3 g, const T* __restrict__ cells,
                                                   const double* __restrict__ edges2, const float* __restrict__ binf,
                                                   float lo2f, float hi2f, unsigned long long* hist) {
    __shared__ unsigned int sh[kHistBins];
    __shared__ float sb[2 * kHistBins + 2];
    for (int b = threadIdx.x; b < kHistBins; b += kHistB3) sh[b] = 0;
    for (int b = threadIdx.x; b < 2 * kHistBins + 2; b += kHistB3) sb[b] = binf[b];
    __syncthreads();
    const float sigf = (float)g.sigma, inv_drf = (float)(1.0 / (kHistDr * g.sigma));
    const unsigned s = blockIdx.x * kHistB3 + threadIdx.x;
    if (s < g.C) {
        const unsigned Q = s / g.cq, r0 = s % g.cq;
        const int ix = (int)(r0 % (unsigned)g.h[0]);
        const unsigned r1 = r0 / (unsigned)g.h[0];
        const int iy = (int)(r1 % (unsigned)g.h[1]), iz = (int)(r1 / (unsigned)g.h[1]);
        const int c3[3] = {2 * ix + (int)(Q & 1), 2 * iy + (int)((Q >> 1) & 1), 2 * iz + (int)(Q >> 2)};
        T px[8], py[8], pz[8];
        ld_cell3(cells, g, s, px, py, pz);
        int n = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) n += px[j] != (T)kEmpty;
        if (n > 0) {
            // binary32 widths and the range of offsets per axis
            float wf[3];
            int lo[3], hi[3];
            const float rlim = (float)((g.sigma + (double)kHistBins * kHistDr * g.sigma) * (1.0 + 1.0e-6));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                wf[a] = g.wf[a];
                float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float v = (float)(a == 0 ? px[j] : (a == 1 ? py[j] : pz[j]));
                    if (j < n) {
                        mn = fminf(mn, v);
                        mx = fmaxf(mx, v);
                    }
                }
                // cell -2 spans [-2w, -w], cell +2 spans [2w, 3w] (margins well
                // above the binary32 rounding of these bounds)
                lo[a] = mn + wf[a] < rlim * (1.0f + 1.0e-5f) ? -2 : -1;
                hi[a] = 2.0f * wf[a] - mx < rlim * (1.0f + 1.0e-5f) ? 2 : 1;
            }
            const double w0 = sizeof(T) == 8 ? g.w[0] : (double)g.wf[0];
            const double w1 = sizeof(T) == 8 ? g.w[1] : (double)g.wf[1];
            const double w2 = sizeof(T) == 8 ? g.w[2] : (double)g.wf[2];
            for (int dz = lo[2]; dz <= hi[2]; ++dz)
                for (int dy = lo[1]; dy <= hi[1]; ++dy)
                    for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                        const unsigned sn = sidx3(g, wrap3(c3[0] + dx, g.m[0]), wrap3(c3[1] + dy, g.m[1]),
                                                  wrap3(c3[2] + dz, g.m[2]));
                        T qx[8], qy[8], qz[8];
                        ld_cell3(cells, g, sn, qx, qy, qz);
                        const float sxf = (float)dx * wf[0], syf = (float)dy * wf[1], szf = (float)dz * wf[2];
                        const bool self = dx == 0 && dy == 0 && dz == 0;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (qx[j] == (T)kEmpty) continue;
                            const float ex = (float)qx[j] + sxf, ey = (float)qy[j] + syf, ez = (float)qz[j] + szf;
                            for (int i = 0; i < n; ++i) {
                                if (self && j == i) continue;   // the sphere itself
                                const T ax = pick8(px, i), ay = pick8(py, i), az = pick8(pz, i);
                                const float fx = (float)ax - ex, fy = (float)ay - ey, fz = (float)az - ez;
                                const float r2f = fx * fx + fy * fy + fz * fz;
                                if (r2f < lo2f || r2f > hi2f) continue;
                                // the bin, decided in binary32 where that is certain
                                int bb = (int)((r2f * rsqrtf(r2f) - sigf) * inv_drf);
                                bb = bb < 0 ? 0 : (bb > kHistBins - 1 ? kHistBins - 1 : bb);
                                if (r2f >= sb[2 * bb] && r2f < sb[2 * bb + 1]) {
                                    atomicAdd(&sh[bb], 1u);
                                    continue;
                                }
                                if (r2f < sb[2 * kHistBins] || r2f >= sb[2 * kHistBins + 1]) continue;
                                hist_pair_exact<T>(ax, ay, az, qx[j], qy[j], qz[j], dx, dy, dz, w0, w1, w2, edges2, sh);
                            }
                        }
                    }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += kHistB3)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// Check of a cell image (snapshot load): occupied slots form a prefix of
// each cell (slot 3 occupied before the secondary half is read), occupied
// coordinates lie in [0, w) on every axis, empty slots hold kEmpty in all
// three coordinates.  out[0] += spheres, out[1] |= 1 on a bad cell.
template <typename T>
__global__ void __launch_bounds__(256) k_check3(G3 g, const T* __restrict__ cells, unsigned long long* out) {
    const unsigned s = blockIdx.x * 256 + threadIdx.x;
    unsigned n = 0;
    bool bad = false;
    if (s < g.C) {
        T x[8], y[8], z[8];
        ld_cell3(cells, g, s, x, y, z);
        bool empty_seen = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (x[j] == (T)kEmpty && y[j] == (T)kEmpty && z[j] == (T)kEmpty) {
                empty_seen = true;
            } else {
                bad |= empty_seen || !(x[j] >= (T)0 && x[j] < Ar3<T>::w(g, 0)) ||
                       !(y[j] >= (T)0 && y[j] < Ar3<T>::w(g, 1)) || !(z[j] >= (T)0 && z[j] < Ar3<T>::w(g, 2));
                ++n;
            }
        }
    }
    const unsigned tot = __reduce_add_sync(0xFFFFFFFFu, n);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(out, (unsigned long long)tot);
    if (bad) atomicOr(out + 1, 1ull);
}

}  // namespace hdmc

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using namespace hdmc;

struct hdmc3_handle {
    G3 g;
    int64_t N;
    double L[3];
    int prec;
    cudaStream_t stream;
    size_t el;                 // bytes per coordinate
    void* cells[2];            // current state and shift target
    int cur;
    Draw3* table;              // kDrawChunk3 sweep draws + 1 extra entry
    Dev3* st;
    unsigned long long* hist;  // kHistBins accumulator
    double* edges2;            // kHistBins + 1 squared bin edges
    float* binf;               // binary32 bin bounds that decide a bin for certain (certified_bins)
    float lo2f, hi2f;
    int64_t samples;
    uint64_t sweeps, shifts;
};

namespace {

int finish3(hdmc3_t* h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_code(e);
    unsigned int err = 0;
    e = cudaMemcpy(&err, &h->st->error, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_code(e);
    return error_code(err);
}

bool make_grid3(const double L[3], double sigma, int m[3], double w[3]) {
    if (!(sigma > 0)) return false;
    for (int a = 0; a < 3; ++a) {
        if (!(L[a] > 0) || !std::isfinite(L[a])) return false;
        const double q = std::floor(L[a] / sigma);
        if (q > 2.0e9) return false;
        m[a] = (int)q;
        m[a] -= m[a] & 1;
        if (m[a] < 4) return false;
        w[a] = L[a] / m[a];
    }
    if ((int64_t)m[0] * m[1] * m[2] >= (int64_t(1) << 32)) return false;
    return (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2] < 4.0 * sigma * sigma;
}

// Face-centred cubic start (same definition as documented in hdmc.h).
bool fcc_positions(int64_t N, const double L[3], double sigma, uint32_t k0, uint32_t k1, std::vector<double>& xyz) {
    int64_t q = 1;
    while (4 * q * q * q < N) ++q;
    if (N < 4 || 4 * q * q * q != N) return false;
    static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    xyz.resize(3 * (size_t)N);
    const double rj = 0.01 * sigma;
    for (int64_t k = 0; k < q; ++k)
        for (int64_t j = 0; j < q; ++j)
            for (int64_t i = 0; i < q; ++i)
                for (int s = 0; s < 4; ++s) {
                    const int64_t p = 4 * ((k * q + j) * q + i) + s;
                    const int64_t b[3] = {i, j, k};
                    WordStream ws(k0, k1, (uint32_t)p, 0xFFFFFFFEu, kDomInit << 28);
                    double u[3];
                    for (;;) {
                        for (int a = 0; a < 3; ++a) {
                            const uint32_t hi = ws.next();
                            const uint32_t lo = ws.next();
                            u[a] = sym52(hi, lo);
                        }
                        if ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2] < 1.0) break;
                    }
                    for (int a = 0; a < 3; ++a) {
                        double x = ((double)b[a] + basis[s][a] + 0.25) * (L[a] / (double)q) + rj * u[a];
                        if (x >= L[a]) x -= L[a];
                        if (x < 0.0) x += L[a];
                        xyz[3 * p + a] = x;
                    }
                }
    return true;
}

// Canonical state (local[(8c+j)*3+a], cnt[c]) of global coordinates.
int bin3(const hdmc3_t* h, const double* xyz, std::vector<double>& loc, std::vector<uint8_t>& cnt) {
    const G3& g = h->g;
    loc.assign((size_t)g.C * kCell3, kEmpty);
    cnt.assign((size_t)g.C, 0);
    for (int64_t p = 0; p < h->N; ++p) {
        int cc[3];
        double l[3];
        for (int a = 0; a < 3; ++a) {
            const double x = xyz[3 * p + a];
            if (!(x >= 0.0 && x <= h->L[a])) return HDMC_EINVAL;
            bin_axis(x, g.w[a], g.m[a], cc[a], l[a]);
            if (h->prec == HDMC_FP32_LOCAL) {
                float f = (float)l[a];
                if (f >= g.wf[a]) f = g.wprevf[a];
                l[a] = f;
            }
        }
        const size_t c = ((size_t)cc[2] * g.m[1] + cc[1]) * g.m[0] + cc[0];
        if (cnt[c] >= kSlots3) return HDMC_EOVERFLOW;
        const int j = cnt[c]++;
        for (int a = 0; a < 3; ++a) loc[(8 * c + j) * 3 + a] = l[a];
    }
    return HDMC_OK;
}

// Overlap test of every sphere against its 27-cell neighbourhood with the
// arithmetic of the sweep.
bool any_overlap3(const hdmc3_t* h, const std::vector<double>& loc, const std::vector<uint8_t>& cnt) {
    const G3& g = h->g;
    for (int cz = 0; cz < g.m[2]; ++cz)
        for (int cy = 0; cy < g.m[1]; ++cy)
            for (int cx = 0; cx < g.m[0]; ++cx) {
                const size_t c = ((size_t)cz * g.m[1] + cy) * g.m[0] + cx;
                for (int i = 0; i < cnt[c]; ++i)
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int n3[3] = {(cx + dx + g.m[0]) % g.m[0], (cy + dy + g.m[1]) % g.m[1],
                                                   (cz + dz + g.m[2]) % g.m[2]};
                                const int dd[3] = {dx, dy, dz};
                                const size_t nc = ((size_t)n3[2] * g.m[1] + n3[1]) * g.m[0] + n3[0];
                                for (int j = 0; j < cnt[nc]; ++j) {
                                    if (dx == 0 && dy == 0 && dz == 0 && i == j) continue;
                                    if (h->prec == HDMC_FP64) {
                                        double e[3];
                                        for (int a = 0; a < 3; ++a)
                                            e[a] = loc[(8 * c + i) * 3 + a] -
                                                   (loc[(8 * nc + j) * 3 + a] + (double)dd[a] * g.w[a]);
                                        if ((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2] < g.sig2) return true;
                                    } else {
                                        float e[3];
                                        for (int a = 0; a < 3; ++a)
                                            e[a] = (float)loc[(8 * c + i) * 3 + a] -
                                                   ((float)loc[(8 * nc + j) * 3 + a] + (float)dd[a] * g.wf[a]);
                                        if (std::fma(e[0], e[0], std::fma(e[1], e[1], std::fma(e[2], e[2], -g.sig2f))) <
                                            0.0f)
                                            return true;
                                    }
                                }
                            }
            }
    return false;
}

// Element index of slot j, coordinate a of the cell with storage index s.
size_t host_slot3(const G3& g, size_t s, int j, int a) {
    return j < 4 ? s * kHalf3 + 4 * a + j : ((size_t)g.C + s) * kHalf3 + 4 * a + (j - 4);
}

void pack3(const hdmc3_t* h, const std::vector<double>& loc, const std::vector<uint8_t>& cnt, std::vector<char>& raw) {
    const G3& g = h->g;
    raw.assign((size_t)g.C * kCell3 * h->el, 0);
    for (int cz = 0; cz < g.m[2]; ++cz)
        for (int cy = 0; cy < g.m[1]; ++cy)
            for (int cx = 0; cx < g.m[0]; ++cx) {
                const size_t c = ((size_t)cz * g.m[1] + cy) * g.m[0] + cx;
                const size_t s = sidx3(g, cx, cy, cz);
                for (int j = 0; j < kSlots3; ++j)
                    for (int a = 0; a < 3; ++a) {
                        const double v = j < cnt[c] ? loc[(8 * c + j) * 3 + a] : kEmpty;
                        char* dst = raw.data() + host_slot3(g, s, j, a) * h->el;
                        if (h->prec == HDMC_FP64) std::memcpy(dst, &v, 8);
                        else {
                            const float f = (float)v;
                            std::memcpy(dst, &f, 4);
                        }
                    }
            }
}

void unpack3(const hdmc3_t* h, const std::vector<char>& raw, std::vector<double>& loc, std::vector<uint8_t>& cnt) {
    const G3& g = h->g;
    loc.assign((size_t)g.C * kCell3, kEmpty);
    cnt.assign((size_t)g.C, 0);
    for (int cz = 0; cz < g.m[2]; ++cz)
        for (int cy = 0; cy < g.m[1]; ++cy)
            for (int cx = 0; cx < g.m[0]; ++cx) {
                const size_t c = ((size_t)cz * g.m[1] + cy) * g.m[0] + cx;
                const size_t s = sidx3(g, cx, cy, cz);
                int n = 0;
                for (int j = 0; j < kSlots3; ++j) {
                    double v[3];
                    for (int a = 0; a < 3; ++a) {
                        const char* src = raw.data() + host_slot3(g, s, j, a) * h->el;
                        if (h->prec == HDMC_FP64) std::memcpy(&v[a], src, 8);
                        else {
                            float f;
                            std::memcpy(&f, src, 4);
                            v[a] = f;
                        }
                    }
                    if (v[0] == kEmpty) break;   // slots fill from 0; a secondary half is valid only after a full primary
                    n = j + 1;
                    for (int a = 0; a < 3; ++a) loc[(8 * c + j) * 3 + a] = v[a];
                }
                cnt[c] = (uint8_t)n;
            }
}

int download3(hdmc3_t* h, std::vector<double>& loc, std::vector<uint8_t>& cnt) {
    int e = finish3(h);
    std::vector<char> raw((size_t)h->g.C * kCell3 * h->el);
    const cudaError_t ce = cudaMemcpy(raw.data(), h->cells[h->cur], raw.size(), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_code(ce);
    unpack3(h, raw, loc, cnt);
    return e;
}

void launch_sub3(hdmc3_t* h, int jd, int k) {
    const unsigned blocks = (h->g.cq + kSubB3 - 1) / kSubB3;
    if (h->prec == HDMC_FP64)
        k_sub3<double><<<blocks, kSubB3, 0, h->stream>>>(h->g, (double*)h->cells[h->cur], h->table, jd, k, h->st);
    else
        k_sub3<float><<<blocks, kSubB3, 0, h->stream>>>(h->g, (float*)h->cells[h->cur], h->table, jd, k, h->st);
}

void launch_shift3(hdmc3_t* h, int jd) {
    const unsigned blocks = (h->g.C + kShiftB3 - 1) / kShiftB3;
    if (h->prec == HDMC_FP64)
        k_shift3<double><<<blocks, kShiftB3, 0, h->stream>>>(h->g, (const double*)h->cells[h->cur],
                                                              (double*)h->cells[1 - h->cur], h->table, jd, h->st);
    else
        k_shift3<float><<<blocks, kShiftB3, 0, h->stream>>>(h->g, (const float*)h->cells[h->cur],
                                                             (float*)h->cells[1 - h->cur], h->table, jd, h->st);
    h->cur = 1 - h->cur;
}

void free3(hdmc3_t* h) {
    if (!h) return;
    cudaFree(h->cells[0]);
    cudaFree(h->cells[1]);
    cudaFree(h->table);
    cudaFree(h->st);
    cudaFree(h->hist);
    cudaFree(h->edges2);
    cudaFree(h->binf);
    delete h;
}

// n sweeps; with events, the mean device time of the sub-sweep and shift
// launches is measured.
int enqueue_sweeps3(hdmc3_t* h, int64_t n, double* ms_sub, double* ms_shift) {
    if (n < 0) return HDMC_EINVAL;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    auto mark = [&](int k) {
        if (!ms_sub && !ms_shift) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, h->stream);
        ev.push_back(e);
        kind.push_back(k);
    };
    for (int64_t done = 0; done < n;) {
        const int cnt = (int)std::min<int64_t>(kDrawChunk3, n - done);
        k_draws3<<<1, kDrawChunk3, 0, h->stream>>>(h->g, h->table, (uint32_t)h->sweeps, cnt, 1);
        for (int j = 0; j < cnt; ++j) {
            for (int k = 0; k < 8; ++k) {
                mark(0);
                launch_sub3(h, j, k);
                mark(-1);
            }
            mark(1);
            launch_shift3(h, j);
            mark(-1);
            h->sweeps += 1;
        }
        done += cnt;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        for (auto x : ev) cudaEventDestroy(x);
        return cuda_code(e);
    }
    if (!ev.empty()) {
        cudaEventSynchronize(ev.back());
        double tot[2] = {0, 0};
        int num[2] = {0, 0};
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            tot[kind[i]] += ms;
            num[kind[i]] += 1;
        }
        for (auto x : ev) cudaEventDestroy(x);
        if (ms_sub) *ms_sub = num[0] ? tot[0] / num[0] : 0.0;
        if (ms_shift) *ms_shift = num[1] ? tot[1] / num[1] : 0.0;
    }
    return HDMC_OK;
}

int set_geometry3(G3& g, const double L[3], double sigma, double d, int nselect, uint64_t seed) {
    int m[3];
    double w[3];
    if (!make_grid3(L, sigma, m, w)) return HDMC_EINVAL;
    if (nselect < 1 || nselect > 255) return HDMC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(d > 0) || !(d < 0.5 * w[a])) return HDMC_EINVAL;
    g = G3{};
    for (int a = 0; a < 3; ++a) {
        g.m[a] = m[a];
        g.h[a] = m[a] / 2;
        g.w[a] = w[a];
        g.wf[a] = (float)w[a];
        g.wprev[a] = std::nextafter(w[a], 0.0);
        g.wprevf[a] = std::nextafter(g.wf[a], 0.0f);
    }
    g.cq = (unsigned)((int64_t)g.h[0] * g.h[1] * g.h[2]);
    g.C = 8u * g.cq;
    g.sigma = sigma;
    g.sig2 = sigma * sigma;
    g.sig2f = (float)(sigma * sigma);
    g.keep2f = (float)(sigma * sigma * (1.0 + 1.0e-3));
    g.band_lo = (float)(sigma * sigma * (1.0 - 0x1p-14));
    g.band_hi = (float)(sigma * sigma * (1.0 + 0x1p-14));
    g.d = d;
    g.df = (float)d;
    g.nsel = nselect;
    g.key0 = (uint32_t)seed;
    g.key1 = (uint32_t)(seed >> 32);
    return HDMC_OK;
}

// ---- snapshots ------------------------------------------------------------------
constexpr char kSnap3Magic[8] = {'H', 'D', 'M', 'C', '3', 'S', 'N', '1'};
constexpr uint32_t kSnap3Version = 1;
constexpr size_t kSnap3Header = 256;

struct Snap3Header {
    char magic[8];
    uint32_t version, precision;
    int64_t N;
    double L[3], sigma, d;
    int32_t nsel, m[3];
    uint32_t key0, key1, flags, pad;
    uint64_t sweeps, shifts;
    int64_t n_samples;
    uint64_t off_state, off_hist, off_cells, cell_bytes, total;
};
static_assert(sizeof(Snap3Header) <= kSnap3Header, "sphere snapshot header");

struct Snap3Layout {
    size_t state, hist, cells, cell_bytes, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Snap3Layout snap3_layout(const hdmc3_t* h) {
    Snap3Layout L;
    L.state = kSnap3Header;
    L.hist = L.state + align256(sizeof(Dev3));
    L.cells = L.hist + align256(sizeof(unsigned long long) * kHistBins);
    L.cell_bytes = (size_t)h->g.C * kCell3 * h->el;
    L.total = L.cells + L.cell_bytes;
    return L;
}

}  // namespace

extern "C" {

size_t hdmc3_snapshot_bytes(const hdmc3_t* h) { return h ? snap3_layout(h).total : 0; }

int hdmc3_save(hdmc3_t* h, void* buf, size_t bytes) {
    if (!h || !buf) return HDMC_EINVAL;
    const Snap3Layout L = snap3_layout(h);
    if (bytes < L.total) return HDMC_EINVAL;
    char* b = static_cast<char*>(buf);
    Snap3Header hd{};
    std::memcpy(hd.magic, kSnap3Magic, sizeof(kSnap3Magic));
    hd.version = kSnap3Version;
    hd.precision = (uint32_t)h->prec;
    hd.N = h->N;
    for (int a = 0; a < 3; ++a) {
        hd.L[a] = h->L[a];
        hd.m[a] = h->g.m[a];
    }
    hd.sigma = h->g.sigma;
    hd.d = h->g.d;
    hd.nsel = h->g.nsel;
    hd.key0 = h->g.key0;
    hd.key1 = h->g.key1;
    hd.flags = h->g.flags;
    hd.sweeps = h->sweeps;
    hd.shifts = h->shifts;
    hd.n_samples = h->samples;
    hd.off_state = L.state;
    hd.off_hist = L.hist;
    hd.off_cells = L.cells;
    hd.cell_bytes = L.cell_bytes;
    hd.total = L.total;
    std::memset(b, 0, L.cells);
    std::memcpy(b, &hd, sizeof(hd));
    const cudaStream_t s = h->stream;
    int e = cuda_code(cudaMemcpyAsync(b + L.state, h->st, sizeof(Dev3), cudaMemcpyDeviceToHost, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(b + L.hist, h->hist, sizeof(unsigned long long) * kHistBins,
                                      cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaMemcpyAsync(b + L.cells, h->cells[h->cur], L.cell_bytes, cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    Dev3 st;
    std::memcpy(&st, b + L.state, sizeof(st));
    return error_code(st.error);
}

int hdmc3_load(hdmc3_t* h, const void* buf, size_t bytes) {
    if (!h || !buf) return HDMC_EINVAL;
    const Snap3Layout L = snap3_layout(h);
    if (bytes < L.total) return HDMC_EINVAL;
    const char* b = static_cast<const char*>(buf);
    Snap3Header hd;
    std::memcpy(&hd, b, sizeof(hd));
    const G3& g = h->g;
    bool same = std::memcmp(hd.magic, kSnap3Magic, sizeof(kSnap3Magic)) == 0 && hd.version == kSnap3Version &&
                hd.precision == (uint32_t)h->prec && hd.N == h->N && hd.sigma == g.sigma &&
                hd.off_state == L.state && hd.off_hist == L.hist && hd.off_cells == L.cells &&
                hd.cell_bytes == L.cell_bytes && hd.total == L.total;
    for (int a = 0; a < 3; ++a) same = same && hd.L[a] == h->L[a] && hd.m[a] == g.m[a];
    if (!same) return HDMC_EINVAL;
    if (hd.nsel < 1 || hd.nsel > 255 || hd.n_samples < 0 || (hd.flags & ~(kNoParticleShuffle | kNoSetShuffle)) != 0)
        return HDMC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(hd.d > 0) || !(hd.d < 0.5 * g.w[a])) return HDMC_EINVAL;
    Dev3 st;
    std::memcpy(&st, b + L.state, sizeof(st));
    if (st.error != 0) return HDMC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(st.origin[a])) return HDMC_EINVAL;
    // cells into the idle half of the double buffer, checked there
    const cudaStream_t s = h->stream;
    void* idle = h->cells[1 - h->cur];
    unsigned long long* res = reinterpret_cast<unsigned long long*>(h->table + kDrawChunk3);  // scratch
    unsigned long long r[2] = {0, 0};
    int e = cuda_code(cudaMemcpyAsync(idle, b + L.cells, L.cell_bytes, cudaMemcpyHostToDevice, s));
    if (!e) e = cuda_code(cudaMemsetAsync(res, 0, 2 * sizeof(unsigned long long), s));
    if (!e) {
        const unsigned blocks = (g.C + 255) / 256;
        if (h->prec == HDMC_FP64) k_check3<double><<<blocks, 256, 0, s>>>(g, (const double*)idle, res);
        else k_check3<float><<<blocks, 256, 0, s>>>(g, (const float*)idle, res);
        e = cuda_code(cudaGetLastError());
    }
    if (!e) e = cuda_code(cudaMemcpyAsync(r, res, sizeof(r), cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    if (r[1] != 0 || r[0] != (unsigned long long)h->N) return HDMC_EINVAL;
    // commit
    e = cuda_code(cudaMemcpyAsync(h->st, &st, sizeof(Dev3), cudaMemcpyHostToDevice, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(h->hist, b + L.hist, sizeof(unsigned long long) * kHistBins,
                                      cudaMemcpyHostToDevice, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    h->cur = 1 - h->cur;
    h->g.d = hd.d;
    h->g.df = (float)hd.d;
    h->g.nsel = hd.nsel;
    h->g.key0 = hd.key0;
    h->g.key1 = hd.key1;
    h->g.flags = hd.flags;
    h->sweeps = hd.sweeps;
    h->shifts = hd.shifts;
    h->samples = hd.n_samples;
    return HDMC_OK;
}

int hdmc3_create(hdmc3_t** out, int64_t N, double Lx, double Ly, double Lz, double sigma, double d, int nselect,
                 uint64_t seed, int precision, const double* xyz, void* stream) {
    if (!out) return HDMC_EINVAL;
    *out = nullptr;
    if (N < 1 || (precision != HDMC_FP64 && precision != HDMC_FP32_LOCAL)) return HDMC_EINVAL;
    hdmc3_t* h = new hdmc3_t();
    h->L[0] = Lx;
    h->L[1] = Ly;
    h->L[2] = Lz;
    int e = set_geometry3(h->g, h->L, sigma, d, nselect, seed);
    if (!e && (int64_t)h->g.C * kSlots3 < N) e = HDMC_EINVAL;
    if (e) {
        delete h;
        return e;
    }
    h->N = N;
    h->prec = precision;
    h->el = precision == HDMC_FP64 ? 8 : 4;
    h->stream = (cudaStream_t)stream;
    std::vector<double> pos;
    if (!xyz) {
        if (!fcc_positions(N, h->L, sigma, h->g.key0, h->g.key1, pos)) {
            delete h;
            return HDMC_EINVAL;
        }
        xyz = pos.data();
    }
    std::vector<double> loc;
    std::vector<uint8_t> cnt;
    e = bin3(h, xyz, loc, cnt);
    if (!e && any_overlap3(h, loc, cnt)) e = HDMC_EOVERLAP;
    if (e) {
        delete h;
        return e;
    }
    std::vector<char> raw;
    pack3(h, loc, cnt, raw);
    const size_t bytes = raw.size();
    cudaError_t ce = cudaMalloc(&h->cells[0], bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&h->cells[1], bytes);
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&h->table, sizeof(Draw3) * (kDrawChunk3 + 1));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&h->st, sizeof(Dev3));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&h->hist, sizeof(unsigned long long) * kHistBins);
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&h->edges2, sizeof(double) * (kHistBins + 1));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&h->binf, sizeof(float) * (2 * kHistBins + 2));
    if (ce == cudaSuccess) ce = cudaMemcpy(h->cells[0], raw.data(), bytes, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(h->st, 0, sizeof(Dev3));
    if (ce == cudaSuccess) ce = cudaMemset(h->hist, 0, sizeof(unsigned long long) * kHistBins);
    double E[kHistBins + 1];
    squared_edges(sigma, E);
    if (ce == cudaSuccess) ce = cudaMemcpy(h->edges2, E, sizeof(E), cudaMemcpyHostToDevice);
    float B[2 * kHistBins + 2];
    certified_bins(sigma, E, B);
    if (ce == cudaSuccess) ce = cudaMemcpy(h->binf, B, sizeof(B), cudaMemcpyHostToDevice);
    // the set-up above ran on the legacy default stream: finish it before
    // work is enqueued on the handle's stream, which need not wait for it
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) {
        free3(h);
        return cuda_code(ce);
    }
    h->g.check = &h->st->error;
    h->lo2f = (float)(E[0] * (1.0 - 1.0e-4));
    h->hi2f = (float)(E[kHistBins] * (1.0 + 1.0e-4));
    h->cur = 0;
    *out = h;
    return HDMC_OK;
}

int hdmc3_sweep(hdmc3_t* h, int64_t n) {
    if (!h) return HDMC_EINVAL;
    return enqueue_sweeps3(h, n, nullptr, nullptr);
}

int hdmc3_profile_sweeps(hdmc3_t* h, int64_t n, double* ms_subsweep, double* ms_shift) {
    if (!h || n < 1) return HDMC_EINVAL;
    double a = 0, b = 0;
    int e = enqueue_sweeps3(h, n, &a, &b);
    if (e) return e;
    if (ms_subsweep) *ms_subsweep = a;
    if (ms_shift) *ms_shift = b;
    return finish3(h);
}

int hdmc3_profile_stages(hdmc3_t* h, int64_t n, double* ms_subsweep, double* ms_shift) {
    if (!h || n < 1) return HDMC_EINVAL;
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return HDMC_ECUDA;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return HDMC_ECUDA;
    }
    double per[3] = {0.0, 0.0, 0.0};
    int e = HDMC_OK;
    for (int stage = 1; stage <= 2 && !e; ++stage) {
        // stage 1: the draws and eight sub-sweeps of each sweep, no shift;
        // stage 2: the draws and the shift of each sweep
        cudaEventRecord(ev[0], h->stream);
        for (int64_t done = 0; done < n;) {
            const int cnt = (int)std::min<int64_t>(kDrawChunk3, n - done);
            k_draws3<<<1, kDrawChunk3, 0, h->stream>>>(h->g, h->table, (uint32_t)h->sweeps, cnt, 1);
            for (int j = 0; j < cnt; ++j) {
                if (stage == 1)
                    for (int k = 0; k < 8; ++k) launch_sub3(h, j, k);
                else
                    launch_shift3(h, j);
                h->sweeps += 1;
            }
            done += cnt;
        }
        cudaEventRecord(ev[1], h->stream);
        e = cuda_code(cudaEventSynchronize(ev[1]));
        float ms = 0.f;
        if (!e) e = cuda_code(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        per[stage] = (double)ms / (double)(n * (stage == 1 ? 8 : 1));
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e) return e;
    if (ms_subsweep) *ms_subsweep = per[1];
    if (ms_shift) *ms_shift = per[2];
    return finish3(h);
}

int hdmc3_shift(hdmc3_t* h) {
    if (!h) return HDMC_EINVAL;
    k_draws3<<<1, 1, 0, h->stream>>>(h->g, h->table + kDrawChunk3, (uint32_t)h->shifts, 1, 0);
    launch_shift3(h, kDrawChunk3);
    h->shifts += 1;
    return cuda_code(cudaGetLastError());
}

int hdmc3_subsweep(hdmc3_t* h, uint32_t sweep, int Q) {
    if (!h || Q < 0 || Q > 7) return HDMC_EINVAL;
    Draw3 d{};
    d.sweep = sweep;
    for (int q = 0; q < 8; ++q) d.perm[q] = (uint8_t)q;
    d.perm[0] = (uint8_t)Q;
    cudaError_t e = cudaMemcpyAsync(h->table + kDrawChunk3, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_code(e);
    e = cudaStreamSynchronize(h->stream);   // d lives on this stack frame
    if (e != cudaSuccess) return cuda_code(e);
    launch_sub3(h, kDrawChunk3, 0);
    return cuda_code(cudaGetLastError());
}

int hdmc3_sample(hdmc3_t* h) {
    if (!h) return HDMC_EINVAL;
    const unsigned blocks = (h->g.C + kHistB3 - 1) / kHistB3;
    if (h->prec == HDMC_FP64)
        k_hist3<double><<<blocks, kHistB3, 0, h->stream>>>(h->g, (const double*)h->cells[h->cur], h->edges2,
                                                            h->binf, h->lo2f, h->hi2f, h->hist);
    else
        k_hist3<float><<<blocks, kHistB3, 0, h->stream>>>(h->g, (const float*)h->cells[h->cur], h->edges2,
                                                           h->binf, h->lo2f, h->hi2f, h->hist);
    h->samples += 1;
    return cuda_code(cudaGetLastError());
}

int hdmc3_pressure(hdmc3_t* h, double* betaP_over_rho, double* g_contact, uint64_t* hist, int64_t* n_samples) {
    if (!h) return HDMC_EINVAL;
    if (h->samples == 0) {
        const int e = hdmc3_sample(h);
        if (e) return e;
    }
    int e = finish3(h);
    unsigned long long hh[kHistBins];
    cudaError_t ce = cudaMemcpy(hh, h->hist, sizeof(hh), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->hist, 0, sizeof(hh), h->stream);
    if (ce != cudaSuccess) return cuda_code(ce);
    const double sigma = h->g.sigma, dr = kHistDr * sigma, c = kFitRange * sigma;
    const double rho = (double)h->N / (h->L[0] * h->L[1] * h->L[2]);
    std::vector<double> t, gv;
    for (int i = 0; i < kHistBins; ++i) {
        const double r0 = sigma + dr * i, r1 = sigma + dr * (i + 1);
        const double v0 = r0 * r0 * r0, v1 = r1 * r1 * r1;
        const double R = 0.75 * (r1 * v1 - r0 * v0) / (v1 - v0);
        if (!(R > sigma && R <= sigma + c)) continue;
        t.push_back((R - sigma) / c);
        gv.push_back((double)hh[i] / ((double)h->samples * (double)h->N * rho * (4.0 * M_PI / 3.0) * (v1 - v0)));
    }
    const double g0 = poly_intercept(t, gv, kFitDegree);
    if (betaP_over_rho) *betaP_over_rho = 1.0 + (2.0 * M_PI / 3.0) * rho * sigma * sigma * sigma * g0;
    if (g_contact) *g_contact = g0;
    if (hist)
        for (int i = 0; i < kHistBins; ++i) hist[i] = hh[i];
    if (n_samples) *n_samples = h->samples;
    h->samples = 0;
    return e;
}

int hdmc3_get_state(hdmc3_t* h, double* local, uint8_t* counts) {
    if (!h || !local || !counts) return HDMC_EINVAL;
    std::vector<double> loc;
    std::vector<uint8_t> cnt;
    const int e = download3(h, loc, cnt);
    if (e && e != HDMC_EOVERFLOW) return e;
    std::memcpy(local, loc.data(), loc.size() * sizeof(double));
    std::memcpy(counts, cnt.data(), cnt.size());
    return e;
}

int hdmc3_positions(hdmc3_t* h, double* xyz) {
    if (!h || !xyz) return HDMC_EINVAL;
    std::vector<double> loc;
    std::vector<uint8_t> cnt;
    int e = download3(h, loc, cnt);
    if (e && e != HDMC_EOVERFLOW) return e;
    Dev3 st;
    const cudaError_t ce = cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_code(ce);
    const G3& g = h->g;
    double w[3], L[3];
    for (int a = 0; a < 3; ++a) {
        w[a] = h->prec == HDMC_FP64 ? g.w[a] : (double)g.wf[a];
        L[a] = h->prec == HDMC_FP64 ? h->L[a] : (double)g.m[a] * w[a];
    }
    int64_t p = 0;
    for (int cz = 0; cz < g.m[2]; ++cz)
        for (int cy = 0; cy < g.m[1]; ++cy)
            for (int cx = 0; cx < g.m[0]; ++cx) {
                const size_t c = ((size_t)cz * g.m[1] + cy) * g.m[0] + cx;
                const int cc[3] = {cx, cy, cz};
                for (int j = 0; j < cnt[c]; ++j) {
                    if (p >= h->N) return HDMC_EOVERFLOW;
                    for (int a = 0; a < 3; ++a) {
                        const double gl = st.origin[a] + ((double)cc[a] * w[a] + loc[(8 * c + j) * 3 + a]);
                        xyz[3 * p + a] = gl - L[a] * std::floor(gl / L[a]);
                    }
                    ++p;
                }
            }
    return e;
}

int hdmc3_counters(hdmc3_t* h, uint64_t out[4]) {
    if (!h || !out) return HDMC_EINVAL;
    const int e = finish3(h);
    Dev3 st;
    const cudaError_t ce = cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_code(ce);
    for (int k = 0; k < 4; ++k) out[k] = st.ctr[k];
    return e;
}

int hdmc3_info(hdmc3_t* h, int32_t m[3], double w[3], double origin[3], uint64_t* sweeps_done,
               uint64_t* shifts_done) {
    if (!h) return HDMC_EINVAL;
    const int e = finish3(h);
    Dev3 st;
    const cudaError_t ce = cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_code(ce);
    for (int a = 0; a < 3; ++a) {
        if (m) m[a] = h->g.m[a];
        if (w) w[a] = h->g.w[a];
        if (origin) origin[a] = st.origin[a];
    }
    if (sweeps_done) *sweeps_done = h->sweeps;
    if (shifts_done) *shifts_done = h->shifts;
    return e;
}

int hdmc3_set_move_size(hdmc3_t* h, double d) {
    if (!h) return HDMC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(d > 0) || !(d < 0.5 * h->g.w[a])) return HDMC_EINVAL;
    h->g.d = d;
    h->g.df = (float)d;
    return HDMC_OK;
}

int hdmc3_set_balance(hdmc3_t* h, int shuffle_particles, int shuffle_sets) {
    if (!h) return HDMC_EINVAL;
    h->g.flags = (shuffle_particles ? 0u : kNoParticleShuffle) | (shuffle_sets ? 0u : kNoSetShuffle);
    return HDMC_OK;
}

int hdmc3_sync(hdmc3_t* h) {
    if (!h) return HDMC_EINVAL;
    return finish3(h);
}

void hdmc3_destroy(hdmc3_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free3(h);
}

}  // extern "C"
