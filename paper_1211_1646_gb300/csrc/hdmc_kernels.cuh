// hdmc_kernels.cuh -- cell-shift, contact-histogram, batched-replica and
// snapshot-check kernels, and the launchers.  Included once by each
// precision's translation unit.
//
// Every floating-point operation that decides an ownership or a histogram
// bin is written with an explicit round-to-nearest operation.
#pragma once

#include "hdmc_common.cuh"
#include "hdmc_subsweep.cuh"

namespace hdmc {

// ---- cell shift: Alg. 4 ----------------------------------------------------------------
// Every disk is translated by -f*ds (equivalently the grid moves by +f*ds).
// One thread per new cell; grid (set row, set column, set).  New cell c = the
// disks of old c that stay inside c (old slot order), then the disks of old
// c+f that leave c+f, re-expressed in c's frame (+f*w).  The ownership test
// is the same computation in the two threads that see a disk, so every disk
// lands in exactly one cell (Sec. 3.2).  A re-expressed value that rounds
// onto the upper edge is clamped below it.
//
// Grid origin O += f*ds (one thread per shift), binary64: ds added or
// subtracted (the same rounding as adding -ds).  Kept out of line so that
// the binary64 instruction stays in that one thread.
static __device__ __noinline__ void add_origin(DevState* __restrict__ st, int ax, int sgn, double ds) {
    st->origin[ax] = sgn > 0 ? __dadd_rn(st->origin[ax], ds) : __dsub_rn(st->origin[ax], ds);
}

// Per-launch constants of the moving coordinate and the evaluation of the
// disks seen by one new cell: stayer() for a disk of old c (does it stay, and
// its new coordinate if it does), migrant() for a disk of old c + f (does it
// leave c + f, and its coordinate in c's frame if it does).  Both apply the
// same ownership test to a disk, so the two threads that see it agree.
template <typename T> struct ShiftParams;

// binary64 path: dp = x - sgn ds; stays iff 0 <= dp < w; a migrant's new
// coordinate dp + sgn w, clamped into [0, w).
template <> struct ShiftParams<double> {
    double sd, w, sw, wprev;
    const SweepDraw* draw;
    __device__ ShiftParams(const Geometry& g, const SweepDraw& r, int ax, int sgn) {
        draw = &r;
        w = ax ? g.wy : g.wx;
        sd = sgn > 0 ? r.ds : -r.ds;
        sw = sgn > 0 ? w : -w;
        wprev = Prm<double>::prev(w);
    }
    __device__ __forceinline__ double origin_ds() const { return draw->ds; }
    __device__ __forceinline__ void stayer(double x, bool& stay, double& v) const {
        v = __dsub_rn(x, sd);
        stay = Prm<double>::ge0(v) && Prm<double>::lt(v, w);
    }
    __device__ __forceinline__ void migrant(double x, bool& leave, double& v) const {
        const double dp = __dsub_rn(x, sd);
        leave = !(Prm<double>::ge0(dp) && Prm<double>::lt(dp, w));
        v = __dadd_rn(dp, sw);
        v = Prm<double>::lt(v, w) ? v : wprev;
        v = Prm<double>::ge0(v) ? v : 0.0;
    }
};

// binary32 rounding of the real number s + t + eta, |eta| <= mu, |s| >= |t|
// (s, t binary32): r = RN32(s + t), and s + t = r + rho exactly (Fast2Sum).
// All reals within mu of s + t round to r when r is positive, not a power
// of two, and rho stays more than mu inside its rounding interval (half an
// ulp on either side); otherwise ok is cleared.
__device__ __forceinline__ float rn32_certified(float s, float t, float mu, bool& ok) {
    const float r = __fadd_rn(s, t);
    const float rho = __fsub_rn(t, __fsub_rn(r, s));
    const uint32_t rb = __float_as_uint(r);
    const float h = __uint_as_float((rb & 0x7F800000u) - (24u << 23));   // half an ulp of r
    ok = (rb & 0x7FFFFFu) != 0u && rb > (25u << 23) && rb < 0x7F800000u && __fadd_rn(fabsf(rho), mu) < h;
    return r;
}

// binary32 path, remapped in binary64 on the binary32 width W = wf:
// dp = RN64(x - sgn ds); stays iff 0 <= dp < W; the stored coordinate is
// RN32(dp) for a stayer and RN32(RN64(dp + sgn W)) for a migrant, clamped
// below wf.  binary64 arithmetic is slow on this GPU, so the result is
// computed in binary32 without rounding error where that is possible and
// certified: sgn ds = d1 + d2 + d3 (d1 = RN32(sgn ds), d2 = RN32(sgn ds -
// d1), |d3| <= 2^-48 ds); s = RN32(x - d1) with its exact error e
// (TwoSum); t = RN32(e - d2); then x - sgn ds = s + t + eta with
// |eta| <= 2^-46 W.  Where s is farther than 2^-20 W from 0 and from W the
// ownership is decided by s, and rn32_certified rounds the stayer's s + t,
// the +f migrant's (s + W) + t (Fast2Sum, exact) or the -f migrant's
// (s - W) + t (s - W exact, Sterbenz) with the bound mu = 2^-43 W on eta,
// the binary32 rounding of the tails and the binary64 roundings of the
// remap.  The rest, about one disk in 10^5, is evaluated with binary64
// instructions; only that branch touches the binary64 constants.
template <> struct ShiftParams<float> {
    float d1, d2, wf, wprev, tau, mu;
    int sgn;
    bool fast;   // the bounds need cell widths far above the binary32 underflow range
    const SweepDraw* draw;
    __device__ ShiftParams(const Geometry& g, const SweepDraw& r, int ax, int sgn_) {
        sgn = sgn_;
        wf = ax ? g.wyf : g.wxf;
        wprev = Prm<float>::prev(wf);
        d1 = sgn > 0 ? r.dsf : -r.dsf;
        d2 = sgn > 0 ? r.dsf2 : -r.dsf2;
        tau = __fmul_rn(wf, 0x1p-20f);
        mu = __fmul_rn(wf, 0x1p-43f);
        fast = wf > 0x1p-60f;
        draw = &r;
    }
    __device__ __forceinline__ double origin_ds() const { return draw->ds; }
    // s = RN32(x - d1) and t: x - sgn ds = s + t + eta; sw = RN32(s - W)
    __device__ __forceinline__ void split(float x, float& s, float& t, float& sw, bool& sure) const {
        s = __fsub_rn(x, d1);
        const float bb = __fsub_rn(s, x);   // TwoSum(x, -d1): s + e = x - d1 exactly
        const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-d1, bb));
        t = __fsub_rn(e, d2);
        sw = __fsub_rn(s, wf);
        sure = fast && fabsf(s) > tau && fabsf(sw) > tau;   // the ownership test is decided by s
    }
    // binary64 instructions.  The conversion of W is a volatile asm, and ds
    // is added or subtracted rather than negated: binary64 operations on the
    // loop invariants would otherwise be hoisted out of this rare branch and
    // issued by every warp (the binary64 pipe is 1/64 of binary32 here).
    __device__ __forceinline__ void exact(float x, bool& stay, float& v) const {
        double W;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(W) : "f"(wf));
        const double xd = (double)x, ds = draw->ds;
        const double dp = sgn > 0 ? __dsub_rn(xd, ds) : __dadd_rn(xd, ds);
        stay = Prm<double>::ge0(dp) && Prm<double>::lt(dp, W);
        v = __double2float_rn(stay ? dp : (sgn > 0 ? __dadd_rn(dp, W) : __dsub_rn(dp, W)));
    }
    __device__ __forceinline__ void stayer(float x, bool& stay, float& v) const {
        float s, t, sw;
        bool sure, ok;
        split(x, s, t, sw, sure);
        stay = s > 0.0f && sw < 0.0f;
        v = rn32_certified(s, t, mu, ok);
        if (!sure || (stay && !ok)) exact(x, stay, v);
        v = v < wf ? v : wprev;   // v >= 0, or -0 from a -0 stayer as the binary64 rule gives
    }
    __device__ __forceinline__ void migrant(float x, bool& leave, float& v) const {
        float s, t, sw;
        bool sure, ok;
        split(x, s, t, sw, sure);
        leave = !(s > 0.0f && sw < 0.0f);
        if (sgn > 0) {   // (s + W) + t, s + W by Fast2Sum (warp-uniform branch)
            const float s2 = __fadd_rn(s, wf);
            v = rn32_certified(s2, __fadd_rn(__fsub_rn(s, __fsub_rn(s2, wf)), t), mu, ok);
        } else {         // (s - W) + t, s - W exact
            v = rn32_certified(sw, t, mu, ok);
        }
        if (!sure || (leave && !ok)) {
            bool stay;
            exact(x, stay, v);
            leave = !stay;
        }
        v = v < wf ? v : wprev;
    }
};

template <typename T>
__device__ __forceinline__ void shift_cells(const Geometry& g, const T* __restrict__ src, T* __restrict__ dst,
                                            const SweepDraw* __restrict__ draw, DevState* __restrict__ st, int bx,
                                            int by, int q) {
    const int hx = bx * kShiftBX + threadIdx.x;
    const int hy = by * kShiftBY + threadIdx.y;
    const int fdir = draw->fdir;
    const int ax = fdir >> 1;
    const int sgn = (fdir & 1) ? -1 : 1;
    const ShiftParams<T> P(g, *draw, ax, sgn);
    if (hx == 0 && hy == 0 && q == 0) add_origin(st, ax, sgn, P.origin_ds());
    if (hx >= g.hx || hy >= g.hy) return;
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    if (cy < g.slo || cy > g.shi) return;   // a strip's halo rows are not its own
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
    for (int j = 0; j < 4; ++j) {   // stayers of old c (occupied slots form a prefix)
        if (Prm<T>::ge0(o.x[j])) {
            bool stay;
            T v;
            P.stayer(ax ? o.y[j] : o.x[j], stay, v);
            const T vx = ax ? o.x[j] : v, vy = ax ? v : o.y[j];
#pragma unroll
            for (int s = 0; s <= j; ++s) {
                r.x[s] = (stay && kept == s) ? vx : r.x[s];
                r.y[s] = (stay && kept == s) ? vy : r.y[s];
            }
            kept += stay;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {   // migrants of old c + f
        if (Prm<T>::ge0(b.x[j])) {
            bool leave;
            T v;
            P.migrant(ax ? b.y[j] : b.x[j], leave, v);
            const T vx = ax ? b.x[j] : v, vy = ax ? v : b.y[j];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                r.x[s] = (leave && kept == s) ? vx : r.x[s];
                r.y[s] = (leave && kept == s) ? vy : r.y[s];
            }
            kept += leave;
        }
    }
    if (kept > 4) atomicOr(&st->error, kErrOverflow);
    store_cell(dst + 8 * idx, r);
}

template <typename T>
__global__ void __launch_bounds__(kShiftBX * kShiftBY)
k_shift(const Geometry g, const T* __restrict__ src, T* __restrict__ dst, const SweepDraw* __restrict__ draw,
        DevState* __restrict__ st) {
    pdl_release();
    pdl_wait();
    // the four sets of one tile are adjacent blocks (set = blockIdx.x & 3), so
    // the old cells a block reads from the neighbouring set are read by that
    // set's block at about the same time: the second read hits L2 even when
    // the state does not fit there
    shift_cells<T>(g, src, dst, draw, st, blockIdx.x >> 2, blockIdx.y, blockIdx.x & 3);
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
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    const bool live = hx < g.hx && hy < g.hy && cy >= g.slo && cy <= g.shi;   // own rows only
    uint32_t* sq = squeue[threadIdx.y];
    Cell<T> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = T(kEmpty);
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

// ---- bond-orientational order psi_6 (Sec. 3.3's order parameter) -------------------------
// Neighbours k of disk j: the other disks closer than r_cut (r_cut <= 2 w, so
// the 5x5 neighbourhood holds them); psi_6(j) = (1/n_j) sum_k z^6 / (|z|^2)^3,
// z = dx + i dy from cell-local coordinates as in the histogram, 0 without
// neighbours.  Pairs in the order dy, dx, slot and every binary64 operation
// explicitly rounded, so psi_6(j) is the same number whatever the launch.
// One thread per cell (grid of the histogram); block sums of
// {re, im, |psi_6|, n} in a fixed order to partial[4 * block].
template <typename T>
__global__ void __launch_bounds__(kHistBX * kHistBY)
k_psi6(const Geometry g, const T* __restrict__ cells, double rc2, double* __restrict__ psi,
       double* __restrict__ partial) {
    __shared__ double red[kHistBY][4];
    const int q = blockIdx.z;
    const int hx = blockIdx.x * kHistBX + threadIdx.x, hy = blockIdx.y * kHistBY + threadIdx.y;
    const bool live = hx < g.hx && hy < g.hy;
    const int cx = 2 * hx + (q & 1), cy = 2 * hy + (q >> 1);
    const double wxd = (double)Prm<T>::wx(g), wyd = (double)Prm<T>::wy(g);
    Cell<T> own;
#pragma unroll
    for (int j = 0; j < 4; ++j) own.x[j] = own.y[j] = T(kEmpty);
    if (live) load_cell_ro(cells + 8 * ((long long)q * g.cq + (long long)hy * g.hx + hx), own);
    double are[4] = {0, 0, 0, 0}, aim[4] = {0, 0, 0, 0};
    int nb[4] = {0, 0, 0, 0};
    if (live) {
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                Cell<T> c;
                load_cell_ro(cells + 8 * storage_index(g, wrap(cx + dx, g.mx), wrap(cy + dy, g.my)), c);
                const double sx = (double)dx * wxd, sy = (double)dy * wyd;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!Prm<T>::ge0(own.x[i])) continue;
                    const double px = (double)own.x[i], py = (double)own.y[i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (!Prm<T>::ge0(c.x[j]) || (dx == 0 && dy == 0 && j == i)) continue;
                        const double ddx = __dsub_rn(px, __dadd_rn((double)c.x[j], sx));
                        const double ddy = __dsub_rn(py, __dadd_rn((double)c.y[j], sy));
                        const double r2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
                        if (!(r2 < rc2)) continue;
                        const double ar = __dsub_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));   // z^2
                        const double ai = __dmul_rn(2.0, __dmul_rn(ddx, ddy));
                        const double br = __dsub_rn(__dmul_rn(ar, ddx), __dmul_rn(ai, ddy));     // z^3
                        const double bi = __dadd_rn(__dmul_rn(ar, ddy), __dmul_rn(ai, ddx));
                        const double zr = __dsub_rn(__dmul_rn(br, br), __dmul_rn(bi, bi));      // z^6
                        const double zi = __dmul_rn(2.0, __dmul_rn(br, bi));
                        const double r6 = __dmul_rn(__dmul_rn(r2, r2), r2);
                        are[i] = __dadd_rn(are[i], __ddiv_rn(zr, r6));
                        aim[i] = __dadd_rn(aim[i], __ddiv_rn(zi, r6));
                        nb[i] += 1;
                    }
                }
            }
    }
    double t[4] = {0, 0, 0, 0};   // re, im, |psi_6|, neighbours of this thread's disks
    const long long cc = (long long)cy * g.mx + cx;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!live || !Prm<T>::ge0(own.x[i])) continue;
        double pr = 0.0, pi = 0.0;
        if (nb[i] > 0) {
            pr = __ddiv_rn(are[i], (double)nb[i]);
            pi = __ddiv_rn(aim[i], (double)nb[i]);
            t[0] = __dadd_rn(t[0], pr);
            t[1] = __dadd_rn(t[1], pi);
            t[2] = __dadd_rn(t[2], __dsqrt_rn(__dadd_rn(__dmul_rn(pr, pr), __dmul_rn(pi, pi))));
        }
        t[3] = __dadd_rn(t[3], (double)nb[i]);
        if (psi) {
            psi[(4 * cc + i) * 2] = pr;
            psi[(4 * cc + i) * 2 + 1] = pi;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) t[k] = __dadd_rn(t[k], __shfl_down_sync(0xffffffffu, t[k], o));
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) red[threadIdx.y][k] = t[k];
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        for (int k = 0; k < 4; ++k) {
            double v = 0.0;
            for (int w = 0; w < kHistBY; ++w) v = __dadd_rn(v, red[w][k]);
            partial[4 * b + k] = v;
        }
    }
}

// ---- batched replicas ------------------------------------------------------------------
// Every stage is one launch over all replicas of a batch: the launch's flat
// block index is mapped to (replica, local block) by a per-stage table, and
// each replica keeps its own geometry, cells, draws, device state,
// counters and histogram.  Replica r's cells start at cell rd.cell_off of
// the arena; its sweep draws of chunk position j sit at draws[j*R + r].
// NSEL > 0: every replica makes NSEL trial moves per cell update.
template <int ROWS, bool TRACK, bool DENSE = false, int NSEL = 0>
static __global__ void __launch_bounds__(32 * ROWS, DENSE ? (16 / ROWS > 0 ? 16 / ROWS : 1) : 20 / ROWS)
k_subsweep_f32_batch(const ReplicaDesc* __restrict__ reps, const unsigned short* __restrict__ map,
                     float* __restrict__ arena, const SweepDraw* __restrict__ draws, int R, int j, int k,
                     unsigned long long* __restrict__ partial, double* __restrict__ msd) {
    __shared__ float2 sdir[kDirRows][32 * ROWS];
    const int r = map[blockIdx.x];
    const ReplicaDesc* rd = reps + r;
    const int local = (int)blockIdx.x - rd->sub_block0;
    const int by = local / rd->sub_gx, bx = local - by * rd->sub_gx;
    subsweep_f32<ROWS, NSEL, TRACK, DENSE>(rd->g, arena + 8 * rd->cell_off, draws + (size_t)j * R + r, k, bx, by,
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
    subsweep_f64<4>(rd->g, arena + 8 * rd->cell_off, draws + (size_t)j * R + r, k, bx, by,
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
    const int q = local & 3, rem = local >> 2;   // the four sets of a tile in adjacent blocks
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
    const dim3 sg = set_grid(c.g, block);
    launch_on(c, k_shift<T>, dim3(4 * sg.x, sg.y, 1), block, c.g, reinterpret_cast<const T*>(src),
              reinterpret_cast<T*>(dst), draw, c.st);
}

template <typename T>
void launch_psi6_t(const LaunchCtx& c, const void* cells, double rc2, double* psi, double* partial) {
    const dim3 block(kHistBX, kHistBY);
    k_psi6<T><<<set_grid(c.g, block), block, 0, c.stream>>>(c.g, reinterpret_cast<const T*>(cells), rc2, psi,
                                                             partial);
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
