// hdmc3_device.cuh -- shared definitions of the three-dimensional (hard
// sphere) kernels: geometry, per-sweep draws, device bookkeeping, the
// set-major cell index and the two-half cell layout, slot shuffles and the
// precision-specific arithmetic of a trial.
//
// Device layout: the cells of one set are contiguous (set-major), row-major
// over the half-resolution grid within a set, as in two dimensions.  A cell
// has 8 slots, filled from slot 0 (an unused slot reads kEmpty), split in two
// halves of 4 slots stored as x0..x3, y0..y3, z0..z3 (48 bytes in binary32,
// 96 in binary64): the primary halves of all C cells, then the secondary
// halves.  A cell holds 1.2 spheres on average at the densities of interest
// and more than 4 in about 0.1 % of the cells, so the kernels read a
// secondary half only when slot 3 is occupied; a secondary half is valid only
// then, and is written only when the cell holds 4 or more.
#pragma once

#include <cstdint>

#include "hdmc_common.cuh"
#include "hdmc_device.cuh"

namespace hdmc {

constexpr int kSlots3 = 8;          // sum of w^2 < 4 sigma^2 => at most 8 centres per cell
constexpr int kCell3 = 3 * kSlots3;  // coordinates per cell
constexpr int kHalf3 = 12;           // coordinates per half cell (4 slots)
constexpr int kSubB3 = 64;          // sub-sweep block: 64 active cells
constexpr int kCand3 = 24;          // gathered neighbour spheres per cell (more: read from global)
constexpr int kShiftB3 = 256;
constexpr int kHistB3 = 128;
constexpr int kDrawChunk3 = 64;     // sweeps per draws launch

struct G3 {
    int m[3];              // cells per axis (even)
    int h[3];              // m/2
    unsigned cq;           // cells per set
    unsigned C;            // all cells
    double w[3];           // widths, binary64
    float wf[3];           // binary32 widths
    double wprev[3];       // largest binary64 below w
    float wprevf[3];       // largest binary32 below wf
    double sigma, sig2;
    float sig2f;
    float keep2f;          // gather threshold sigma^2 (1 + 1e-3), binary32
    float band_lo, band_hi;   // sigma^2 (1 -+ 2^-14): binary32 pair tests outside decide (binary64 mode)
    double d;
    float df;
    int nsel;
    uint32_t key0, key1;
    uint32_t flags;        // kNoParticleShuffle | kNoSetShuffle
    unsigned int* check;   // builds with -DHDMC_CHECK: device word that collects failed index checks
};

struct alignas(8) Draw3 {
    uint32_t sweep;        // counter word 0 of the cell streams
    int32_t fdir;          // 2*axis + (1 for the negative direction)
    uint8_t perm[8];       // set of sub-sweep k
    double ds;
};

struct Dev3 {
    unsigned long long ctr[4];   // trials, accepted, left the cell, overlap
    double origin[3];
    unsigned int error;          // bit 0: a cell received more than 8 spheres
    unsigned int pad;
};

__host__ __device__ inline unsigned sidx3(const G3& g, int cx, int cy, int cz) {
    const unsigned q = (unsigned)((cx & 1) + 2 * (cy & 1) + 4 * (cz & 1));
    return (unsigned)checked_cell(g.check,
                                  q * g.cq + ((unsigned)(cz >> 1) * (unsigned)g.h[1] + (unsigned)(cy >> 1)) *
                                                 (unsigned)g.h[0] + (unsigned)(cx >> 1),
                                  g.C);
}

__device__ __forceinline__ uint32_t factorial8(int n) {
    uint32_t f = 1;
#pragma unroll
    for (int k = 2; k <= 8; ++k) f = k <= n ? f * (uint32_t)k : f;
    return f;
}

// Precision-specific arithmetic; each form is the one the serial reference
// evaluates (binary64: plain operations; binary32: fma where it writes fma).
template <typename T> struct Ar3;
template <> struct Ar3<double> {
    __device__ static double w(const G3& g, int a) { return g.w[a]; }
    __device__ static double trial(const G3& g, double x, double u) { return x + g.d * u; }
    __device__ static bool hit(const G3& g, double dx, double dy, double dz) {
        return (dx * dx + dy * dy) + dz * dz < g.sig2;
    }
};
template <> struct Ar3<float> {
    __device__ static float w(const G3& g, int a) { return g.wf[a]; }
    __device__ static float trial(const G3& g, float x, float u) { return fmaf(g.df, u, x); }
    __device__ static bool hit(const G3& g, float dx, float dy, float dz) {
        return fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, -g.sig2f))) < 0.0f;
    }
};

template <typename T>
__device__ __forceinline__ T pick8(const T (&v)[8], int i) {
    T r = v[0];
#pragma unroll
    for (int j = 1; j < 8; ++j) r = i == j ? v[j] : r;
    return r;
}

template <typename T>
__device__ __forceinline__ void put8(T (&v)[8], int i, T x) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = i == j ? x : v[j];
}

// Swap slots J and r (r <= J) of the three coordinate arrays.
template <int J, typename T>
__device__ __forceinline__ void swap_slot3(T (&x)[8], T (&y)[8], T (&z)[8], int r) {
    const T ax = pick8(x, r), ay = pick8(y, r), az = pick8(z, r);
#pragma unroll
    for (int s = 0; s < J; ++s) {
        x[s] = s == r ? x[J] : x[s];
        y[s] = s == r ? y[J] : y[s];
        z[s] = s == r ? z[J] : z[s];
    }
    x[J] = ax;
    y[J] = ay;
    z[J] = az;
}

// Fisher-Yates decode of k in [0, n!): for j = n-1 down to 1 swap slots j and
// k mod (j+1), then k /= (j+1).
template <typename T>
__device__ __forceinline__ void shuffle3(T (&x)[8], T (&y)[8], T (&z)[8], int n, uint32_t k) {
#define HDMC3_STEP(J)                                        \
    if (J < n) {                                             \
        const int r = (int)(k % (uint32_t)(J + 1));          \
        k /= (uint32_t)(J + 1);                              \
        swap_slot3<J>(x, y, z, r);                           \
    }
    HDMC3_STEP(7) HDMC3_STEP(6) HDMC3_STEP(5) HDMC3_STEP(4) HDMC3_STEP(3) HDMC3_STEP(2) HDMC3_STEP(1)
#undef HDMC3_STEP
}

__device__ __forceinline__ int wrap3(int c, int m) { return c < 0 ? c + m : (c >= m ? c - m : c); }

// Half-cell loads and stores: 4 slots of one coordinate are 16 bytes
// (binary32, one 128-bit access) or 32 bytes (binary64, two).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// The 4 slots of one half cell (at p) into slots OFF..OFF+3.
template <int OFF, typename T>
__device__ __forceinline__ void ld_half3(const T* p, T (&x)[8], T (&y)[8], T (&z)[8]) {
    T a[4], b[4], c[4];
    ld4(p, a);
    ld4(p + 4, b);
    ld4(p + 8, c);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[OFF + i] = a[i];
        y[OFF + i] = b[i];
        z[OFF + i] = c[i];
    }
}

__device__ __forceinline__ size_t primary3(unsigned s) { return (size_t)s * kHalf3; }
__device__ __forceinline__ size_t secondary3(const G3& g, unsigned s) { return ((size_t)g.C + s) * kHalf3; }

// Completes a cell whose primary half is in slots 0..3: reads the secondary
// half when slot 3 is occupied, else marks slots 4..7 empty.
template <typename T>
__device__ __forceinline__ void ld_rest3(const T* cells, const G3& g, unsigned s, T (&x)[8], T (&y)[8], T (&z)[8]) {
    if (x[3] != (T)kEmpty) {
        ld_half3<4>(cells + secondary3(g, s), x, y, z);
    } else {
#pragma unroll
        for (int i = 4; i < 8; ++i) x[i] = y[i] = z[i] = (T)kEmpty;
    }
}

template <typename T>
__device__ __forceinline__ void ld_cell3(const T* cells, const G3& g, unsigned s, T (&x)[8], T (&y)[8], T (&z)[8]) {
    ld_half3<0>(cells + primary3(s), x, y, z);
    ld_rest3(cells, g, s, x, y, z);
}

// Writes the primary half, and the secondary half when `full` (4 or more
// spheres: readers then take slot 3 as occupied and read it).
template <typename T>
__device__ __forceinline__ void st_cell3(T* cells, const G3& g, unsigned s, const T (&x)[8], const T (&y)[8],
                                         const T (&z)[8], bool full) {
    T* p = cells + primary3(s);
    st4(p, x);
    st4(p + 4, y);
    st4(p + 8, z);
    if (full) {
        T* q = cells + secondary3(g, s);
        st4(q, x + 4);
        st4(q + 4, y + 4);
        st4(q + 8, z + 4);
    }
}

// Slot j of cell s (coordinate a at offset 4a); slots 4..7 may be read only
// when slot 3 is occupied.
template <typename T>
__device__ __forceinline__ const T* slot3(const T* cells, const G3& g, unsigned s, int j) {
    return j < 4 ? cells + primary3(s) + j : cells + secondary3(g, s) + (j - 4);
}

}  // namespace hdmc
