// hdmc_noalloc.cu -- contact histogram that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or a memory-capped process, plugins that may not
// own GPU allocations, or code paths where an allocation could fail or
// stall.  hdmc_histogram_noalloc serves them: it reads a caller-owned device
// copy of a configuration and returns the contact histogram in host memory.
// Its only device scratch (the bin accumulator) is a file-scope array of
// HDMC_NOALLOC_MAX_BINS 64-bit counters, which every GPU that loads this
// library holds until the process exits.  All calls share that array and it
// keeps the last call's counts, so each call clears it first, and calls that
// overlap on the GPU (several streams or host threads at once) race on it.
#include <mutex>

#include "hdmc.h"
#include "hdmc_kernels.cuh"

namespace hdmc {
namespace {

constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned long long g_noalloc_hist[HDMC_NOALLOC_MAX_BINS];

// Device address of g_noalloc_hist on each device, looked up on the first
// call made with that device current (host code may not use the array's name
// as an address: on the host it is only a stand-in for the device symbol).
// cudaDeviceReset reloads the module, which may move the array: the cached
// address is then stale, so this entry point is not for processes that reset
// a device they have used it on.
void* g_noalloc_ptr[kMaxDevices];
std::mutex g_noalloc_mu;

int noalloc_scratch(int dev, unsigned long long** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_hist) != cudaSuccess || !p) return HDMC_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = reinterpret_cast<unsigned long long*>(g_noalloc_ptr[dev]);
    return HDMC_OK;
}

// Same pair rule as k_hist (ordered pairs over the 5x5 neighbourhood, exact
// binary64 r^2 against the squared bin edges, conservative binary32
// candidate selection), reading cells in canonical order c = cy*mx + cx with
// slot j of cell c at local[(4c+j)*2], local[(4c+j)*2+1]; a slot is
// occupied iff its x is >= 0, in the own cell and in every neighbour, so an
// empty slot may hold any negative x.
__global__ void __launch_bounds__(256)
k_hist_canonical(const double* __restrict__ local, int mx, int my, double wx, double wy, double sigma, int nbins,
                 double dr, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int sh[HDMC_NOALLOC_MAX_BINS];
    __shared__ double sE[HDMC_NOALLOC_MAX_BINS + 1];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int b = tid; b < nbins; b += blockDim.x * blockDim.y) sh[b] = 0u;
    for (int b = tid; b <= nbins; b += blockDim.x * blockDim.y) {
        const double e = __dadd_rn(sigma, __dmul_rn((double)b, dr));
        sE[b] = __dmul_rn(e, e);
    }
    __syncthreads();
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    const bool live = cx < mx && cy < my;
    auto load = [&](int x, int y, Cell<double>& c) {
        const double2* p = reinterpret_cast<const double2*>(local + 8 * ((long long)y * mx + x));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double2 v = __ldg(p + j);
            c.x[j] = v.x;
            c.y[j] = v.y;
        }
    };
    Cell<double> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = kEmpty;
    if (live) load(cx, cy, own);
    if (__any_sync(0xffffffffu, own.x[0] >= 0.0)) {
        const float rmax = (float)(sigma + (double)nbins * dr);
        const float thr = rmax * rmax * 1.001f;
        const float sigf = (float)sigma, inv_drf = (float)(1.0 / dr);
        const float wxf = (float)wx, wyf = (float)wy;
        float ox[4], oy[4];
        uint32_t occupied = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ox[i] = approx_f32(own.x[i]);
            oy[i] = approx_f32(own.y[i]);
            occupied |= own.x[i] >= 0.0 ? (0xFu << (4 * i)) : 0u;
        }
        const f2x nt = pk(-thr, -thr);
        for (int dy = -2; dy <= 2; ++dy) {
            for (int dx = -2; dx <= 2; ++dx) {
                Cell<double> c;
#pragma unroll
                for (int j = 0; j < 4; ++j) c.x[j] = c.y[j] = kEmpty;
                if (live) load(wrap(cx + dx, mx), wrap(cy + dy, my), c);
                const float sxf = (float)dx * wxf, syf = (float)dy * wyf;
                const f2x qx01 = add2(pk(approx_f32(c.x[0]), approx_f32(c.x[1])), pk(sxf, sxf));
                const f2x qx23 = add2(pk(approx_f32(c.x[2]), approx_f32(c.x[3])), pk(sxf, sxf));
                const f2x qy01 = add2(pk(approx_f32(c.y[0]), approx_f32(c.y[1])), pk(syf, syf));
                const f2x qy23 = add2(pk(approx_f32(c.y[2]), approx_f32(c.y[3])), pk(syf, syf));
                uint32_t cand = 0, nocc = 0;   // nocc: occupied slots j of the neighbour, bits 4i + j
#pragma unroll
                for (int j = 0; j < 4; ++j) nocc |= c.x[j] >= 0.0 ? (0x1111u << j) : 0u;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const f2x tx2 = pk(ox[i], ox[i]), ty2 = pk(oy[i], oy[i]);
                    f2x z = zpair(tx2, ty2, qx01, qy01, nt);
                    cand |= ((lo32(z) >> 31) << (4 * i)) | ((hi32(z) >> 31) << (4 * i + 1));
                    z = zpair(tx2, ty2, qx23, qy23, nt);
                    cand |= ((lo32(z) >> 31) << (4 * i + 2)) | ((hi32(z) >> 31) << (4 * i + 3));
                }
                cand &= occupied & nocc;
                if (dx == 0 && dy == 0) cand &= ~0x8421u;
                while (cand) {
                    const int b = __ffs(cand) - 1;
                    cand &= cand - 1;
                    const int i = b >> 2, j = b & 3;
                    const double ex = __dadd_rn(pick(c.x, j), (double)dx * wx);
                    const double ey = __dadd_rn(pick(c.y, j), (double)dy * wy);
                    const double ddx = __dsub_rn(pick(own.x, i), ex), ddy = __dsub_rn(pick(own.y, i), ey);
                    const double r2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                    if (r2 >= sE[0] && r2 < sE[nbins]) {
                        const float r2f = approx_f32(r2);
                        int bb = (int)((r2f * rsqrtf(r2f) - sigf) * inv_drf);
                        bb = bb < 0 ? 0 : (bb > nbins - 1 ? nbins - 1 : bb);
                        while (bb > 0 && r2 < sE[bb]) --bb;
                        while (bb < nbins - 1 && r2 >= sE[bb + 1]) ++bb;
                        atomicAdd(&sh[bb], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int b = tid; b < nbins; b += blockDim.x * blockDim.y)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

}  // namespace
}  // namespace hdmc

extern "C" int hdmc_histogram_noalloc(const double* dev_local, int32_t mx, int32_t my, double wx, double wy,
                                      double sigma, int32_t nbins, double dr, uint64_t* hist, void* stream) {
    using namespace hdmc;
    if (!dev_local || !hist) return HDMC_EINVAL;
    // the kernel reads the cells with 16-byte loads
    if ((uintptr_t)dev_local % 16 != 0) return HDMC_EINVAL;
    if (nbins < 1 || nbins > HDMC_NOALLOC_MAX_BINS) return HDMC_EINVAL;
    if (mx < 4 || my < 4 || !(sigma > 0) || !(dr > 0) || !(wx > 0) || !(wy > 0)) return HDMC_EINVAL;
    // two rings of cells must reach the largest distance counted
    if (!(sigma + (double)nbins * dr <= 2.0 * wx) || !(sigma + (double)nbins * dr <= 2.0 * wy)) return HDMC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HDMC_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return HDMC_EINVAL;
    unsigned long long* scratch = nullptr;
    int e = noalloc_scratch(dev, &scratch);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)nbins, s) != cudaSuccess) return HDMC_ECUDA;
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((mx + 31) / 32), (unsigned)((my + 7) / 8));
    k_hist_canonical<<<grid, block, 0, s>>>(dev_local, mx, my, wx, wy, sigma, nbins, dr, scratch);
    if (cudaGetLastError() != cudaSuccess) return HDMC_ECUDA;
    if (cudaMemcpyAsync(hist, scratch, sizeof(unsigned long long) * (size_t)nbins, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return HDMC_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? HDMC_OK : HDMC_ECUDA;
}
