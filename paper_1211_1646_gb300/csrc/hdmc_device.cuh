// hdmc_device.cuh -- shared definitions of the CUDA hard-disk Monte Carlo
// library: geometry, per-sweep draws, the counter-based random streams and
// the device-resident bookkeeping.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by
// the 64-bit seed.  Every random decision of the method reads its own
// stream, block b of which is Philox(key, (c0, c1, c2, b)):
//   sweep-level draws of sweep s (Alg. 1: set order, shift):
//                      (s, 0xFFFFFFFF, 2<<28)
//   trial stream of the update of cell c in sweep s, set Q (Alg. 1:
//   shuffle draw, trial directions):
//                      (s, c, (1<<28)|(Q<<24))
//   shuffle stream of that update (binary64 shuffles; binary32 fallback):
//                      (s, c, (0<<28)|(Q<<24))
//   start jitter of disk p:  (p, 0xFFFFFFFE, 3<<28)
//   explicit extra shift k:  (k, 0xFFFFFFFF, 4<<28)
// with c = cy*mx + cx the canonical cell number.  Because the streams are
// counter-based, the cells of one set can run in any order on any number of
// threads and still give one fixed result (the paper's Saru hash plays the
// same role in Alg. 2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hdmc {

constexpr int kSlots = 4;                 // w < sqrt(2) sigma => at most 4 centres per cell (Fig. 3)
constexpr double kEmpty = -1.0e4;         // coordinate of an unused slot (the paper uses (-10,-10))
constexpr int kHistBins = 200;            // contact histogram: 200 bins ...
constexpr double kHistDr = 1.0e-4;        // ... of 1e-4 sigma (Sec. 4)
constexpr double kFitRange = 0.02;        // fit range c = 0.02 sigma (Sec. 4)
constexpr int kFitDegree = 5;             // polynomial degree (Sec. 4)

constexpr uint32_t kDomShuffle = 0u, kDomTrial = 1u, kDomSweep = 2u, kDomInit = 3u, kDomShift = 4u;

constexpr int kHistBX = 32, kHistBY = 8;     // histogram block: 32 set columns x 8 set rows of one set
constexpr int kShiftBX = 64, kShiftBY = 4;   // shift block: 64 set columns x 4 set rows of one set

// Geometry and move parameters, passed by value to every kernel.
struct Geometry {
    int mx, my;            // cells per axis, both even
    int hx, hy;            // mx/2, my/2: cells per set row / per set column
    long long cq;          // cells per checkerboard set = hx*hy
    long long C;           // mx*my
    double wx, wy;         // cell widths (binary64)
    float wxf, wyf;        // binary32 cell widths (FP32 path)
    double sigma, sig2;    // sigma, sigma*sigma
    float sig2f;           // binary32 rounding of sigma*sigma
    double d;              // maximum trial displacement
    float df;              // its binary32 rounding
    int nsel;              // trial moves per cell and sub-sweep (n_M)
    uint32_t key0, key1;   // Philox key = seed
    uint32_t flags;        // kNoParticleShuffle | kNoSetShuffle (Table 1 controls); 0 = the method
    unsigned int* check;   // builds with -DHDMC_CHECK: device word that collects failed index checks
    // Rows of a strip of a larger grid (spatial decomposition, Sec. 6); a
    // whole system has row0 = 0 and both ranges [0, my-1].
    int row0;              // global cell row of row 0 (random streams use global cell numbers)
    int ylo, yhi;          // rows whose cells make trial moves
    int slo, shi;          // rows the shift writes and the contact histogram counts
    int dense;             // cells hold 1.3 disks or more on average (binary32 sub-sweep variant)
};

// Device error word bits: a cell received more than its slots (bit 0); a
// computed cell index fell outside the grid (bit 1, builds with -DHDMC_CHECK
// only, which check every cell index the kernels compute and replace a bad
// one by 0 so that no access leaves the buffer).
constexpr uint32_t kErrOverflow = 1u, kErrIndex = 2u;

// Index check of a -DHDMC_CHECK build (no code otherwise).
__host__ __device__ __forceinline__ long long checked_cell(unsigned int* check, long long idx, long long limit) {
#if defined(HDMC_CHECK) && defined(__CUDA_ARCH__)
    if (idx < 0 || idx >= limit) {
        if (check) atomicOr(check, kErrIndex);
        return 0;
    }
#else
    (void)check;
    (void)limit;
#endif
    return idx;
}

// Balance controls of Table 1 (Sec. 2.4): skip the shuffle of the disks of a
// cell, or take the checkerboard sets in the fixed order 0, 1, 2, 3.  The
// random streams are consumed exactly as with the controls off.
constexpr uint32_t kNoParticleShuffle = 1u, kNoSetShuffle = 2u;

// Draws of one sweep (Alg. 1): set order, shift direction and distance.
struct alignas(16) SweepDraw {
    uint32_t sweep;        // counter word 0 of the sweep's cell streams
    int32_t fdir;          // 0:+x 1:-x 2:+y 3:-y
    uint8_t perm[4];       // checkerboard set of sub-sweep k
    float dsf;             // binary32 rounding of ds
    double ds;             // shift distance, uniform in [0, w/2) along f's axis
    float dsf2;            // binary32 rounding of ds - dsf (ds = dsf + dsf2 within 2^-48 ds)
    uint32_t pad[3];
};

// Device-resident bookkeeping, advanced by the kernels themselves so that a
// recorded CUDA graph of many sweeps can be replayed without host updates.
struct DevState {
    unsigned long long sweep_next;   // index of the next sweep to draw
    unsigned long long shift_next;   // index of the next explicit shift to draw
    double origin[2];                // accumulated grid origin (sum of f*ds)
    unsigned int error;              // bit 0: a cell received more than 4 disks
    unsigned int pad[3];
};

// One replica of a batch: its geometry, where its cells start in the batch
// arena, and its share of each stage's launch (blocks of one replica are
// contiguous in the flat block index).
struct ReplicaDesc {
    Geometry g;
    long long cell_off;   // first cell of the replica in the arena
    long long part_off;   // first sub-sweep counter slot of the replica
    int sub_gx, sub_block0;           // sub-sweep: blocks per set row, first flat block
    int sh_gx, sh_gy, sh_block0;      // shift: blocks per set row / column, first flat block
    int hi_gx, hi_gy, hi_block0;      // histogram: same
};

// Cell storage: the cells of one checkerboard set are contiguous (set-major),
// row-major within the set on the half-resolution grid, so the active cells of
// a sub-sweep form one dense range and a warp reads 32 consecutive cells.
// This generalises Alg. 3 (even/odd x contiguous) to both axes.
__host__ __device__ inline long long storage_index(const Geometry& g, int cx, int cy) {
    const int q = (cx & 1) + 2 * (cy & 1);
    return checked_cell(g.check, (long long)q * g.cq + (long long)(cy >> 1) * g.hx + (cx >> 1), g.C);
}

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Sequential 32-bit words of one stream.
struct WordStream {
    uint32_t k0, k1;
    uint4 ctr;
    uint4 buf;
    int pos;
    __host__ __device__ WordStream(uint32_t key0, uint32_t key1, uint32_t c0, uint32_t c1, uint32_t c2)
        : k0(key0), k1(key1), ctr(make_uint4(c0, c1, c2, 0u)), buf(make_uint4(0, 0, 0, 0)), pos(4) {}
    __host__ __device__ uint32_t next() {
        if (pos == 4) {
            buf = philox4x32_10(ctr, k0, k1);
            ctr.w += 1u;
            pos = 0;
        }
        const uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        ++pos;
        return w;
    }
    // Uniform integer in [0, range): Lemire's multiply-high with exact
    // rejection of low halves below 2^32 mod range.
    __host__ __device__ uint32_t bounded(uint32_t range) {
        for (;;) {
            const uint64_t m = (uint64_t)next() * range;
            const uint32_t lo = (uint32_t)m;
            if (lo >= range) return (uint32_t)(m >> 32);        // lo >= range > 2^32 mod range
            const uint32_t thr = (0u - range) % range;
            if (lo >= thr) return (uint32_t)(m >> 32);
        }
    }
};

// Odd multiples of 2^-52 in (-1,1): exact mirror symmetry u(~w) = -u(w).
__host__ __device__ inline double sym52(uint32_t hi, uint32_t lo) {
    const uint64_t k = (((uint64_t)hi << 32) | lo) >> 12;
    const int64_t m = (int64_t)(2 * k + 1) - ((int64_t)1 << 52);
    return (double)m * 0x1p-52;
}

__host__ __device__ inline double unif53(uint32_t hi, uint32_t lo) {
    const uint64_t k = (((uint64_t)hi << 32) | lo) >> 11;
    return (double)k * 0x1p-53;
}

// Sweep-level draws (Alg. 1): Fisher-Yates order of the four sets, shift
// direction f in {+x,-x,+y,-y}, distance uniform in [0, w/2) along f's axis.
__host__ __device__ inline SweepDraw make_draw(const Geometry& g, uint32_t index, uint32_t domain, bool with_perm) {
    WordStream s(g.key0, g.key1, index, 0xFFFFFFFFu, domain << 28);
    SweepDraw r;
    int p[4] = {0, 1, 2, 3};
    if (with_perm) {
        for (int j = 3; j >= 1; --j) {
            const int k = (int)s.bounded((uint32_t)(j + 1));
            const int t = p[j];
            p[j] = p[k];
            p[k] = t;
        }
    }
    if (g.flags & kNoSetShuffle)
        for (int q = 0; q < 4; ++q) p[q] = q;
    r.fdir = (int32_t)s.bounded(4u);
    const uint32_t hi = s.next(), lo = s.next();
    const double w = (r.fdir >> 1) ? g.wy : g.wx;
    r.ds = unif53(hi, lo) * (0.5 * w);
    r.dsf = (float)r.ds;
    r.sweep = index;
    for (int q = 0; q < 4; ++q) r.perm[q] = (uint8_t)p[q];
    r.dsf2 = (float)(r.ds - (double)r.dsf);
    r.pad[0] = r.pad[1] = r.pad[2] = 0;
    return r;
}

// ---------------------------------------------------------------------------
// Kernel launchers (one translation unit per precision)
// ---------------------------------------------------------------------------
struct LaunchCtx {
    Geometry g;
    cudaStream_t stream;
    bool pdl = false;              // launch as a programmatic dependent of the previous kernel
    DevState* st;
    unsigned long long* partial;   // per-block trial counters, 4 per sub-sweep block
    unsigned long long* hist;      // contact histogram accumulator (kHistBins)
    const double* edges2;          // squared bin edges (sigma + k dr)^2, k = 0..kHistBins
};

// Launches kernel<<<grid, block>>>(args) on c.stream; with c.pdl, as a
// programmatic dependent launch: its blocks may be scheduled while the
// previous kernel of the stream finishes, and wait (griddepcontrol.wait, at
// the top of every such kernel) for its completion before reading anything.
template <typename... P, typename... A>
inline void launch_on(const LaunchCtx& c, void (*kernel)(P...), dim3 grid, dim3 block, A... args) {
    if (!c.pdl) {
        kernel<<<grid, block, 0, c.stream>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

void launch_draws(const LaunchCtx& c, SweepDraw* table, int count, bool sweep_mode);
void launch_draws_batch(cudaStream_t s, const ReplicaDesc* reps, DevState* sts, SweepDraw* table, int R, int count);
// Trial-counter tiles of the sub-sweeps: 32 set columns x kCounterRows set
// rows, one slot of 4 counters each; the sub-sweep kernels run one-row
// blocks, and the blocks of a tile add into its slot.
constexpr int kCounterRows = 4;
dim3 subsweep_grid(const Geometry& g);

void launch_subsweep_f64(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k);
void launch_shift_f64(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw);
void launch_hist_f64(const LaunchCtx& c, const void* cells);
void launch_psi6_f64(const LaunchCtx& c, const void* cells, double rc2, double* psi, double* partial);
void launch_check_f64(const LaunchCtx& c, const void* cells, unsigned long long* out);

void launch_subsweep_f32(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k);

// Batched stages (one launch over all R replicas).
struct BatchCtx {
    cudaStream_t stream;
    const ReplicaDesc* reps;
    const unsigned short* sub_map;
    const unsigned short* sh_map;
    const unsigned short* hi_map;
    int sub_blocks, sh_blocks, hi_blocks;
    int R;
    int rows;                      // sub-sweep block height (binary32): 2, 4 or 8
    bool dense;                    // every replica has crowded cells (Geometry::dense): dense binary32 kernel
    int nsel;                      // n_M of every replica, or 0 if they differ
    DevState* sts;
    unsigned long long* partial;
    unsigned long long* hist;      // R x kHistBins
    const double* edges2;
    double* msd;                   // R net squared displacements (tracking launches)
};
void launch_subsweep_f32_batch(const BatchCtx& c, void* arena, const SweepDraw* draws, int j, int k, bool track);
void launch_subsweep_f64_batch(const BatchCtx& c, void* arena, const SweepDraw* draws, int j, int k);
void launch_shift_batch(const BatchCtx& c, int prec, const void* src, void* dst, const SweepDraw* draws, int j);
void launch_hist_batch(const BatchCtx& c, int prec, const void* arena);
void launch_shift_f32(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw);
void launch_hist_f32(const LaunchCtx& c, const void* cells);
void launch_psi6_f32(const LaunchCtx& c, const void* cells, double rc2, double* psi, double* partial);
unsigned psi6_blocks(const Geometry& g);   // blocks of one psi_6 launch
void launch_check_f32(const LaunchCtx& c, const void* cells, unsigned long long* out);

}  // namespace hdmc
