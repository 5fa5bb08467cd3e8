// Binary32 cell-local coordinates (HDMC_FP32_LOCAL).
#include "hdmc_kernels.cuh"

namespace hdmc {
void launch_subsweep_f32(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k) {
    float* a = reinterpret_cast<float*>(cells);
    // blocks of two set rows of 32 cells: in-step faster than one-row blocks
    // (fewer blocks to schedule) and as fast as four-row blocks
    const dim3 grid((unsigned)((c.g.hx + 31) / 32), (unsigned)((c.g.hy + 1) / 2));
    if (c.g.dense) {   // cells that often hold three or four disks
        if (c.g.nsel == 4)
            launch_on(c, k_subsweep_f32<2, 4, true>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
        else if (c.g.nsel == 8)
            launch_on(c, k_subsweep_f32<2, 8, true>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
        else
            launch_on(c, k_subsweep_f32<2, 0, true>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
    } else if (c.g.nsel == 4) {
        launch_on(c, k_subsweep_f32<2, 4>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
    } else if (c.g.nsel == 8) {
        launch_on(c, k_subsweep_f32<2, 8>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
    } else {
        launch_on(c, k_subsweep_f32<2, 0>, grid, dim3(32, 2), c.g, a, draw, k, c.partial);
    }
}
void launch_shift_f32(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw) {
    launch_shift_t<float>(c, src, dst, draw);
}
void launch_hist_f32(const LaunchCtx& c, const void* cells) { launch_hist_t<float>(c, cells); }
void launch_psi6_f32(const LaunchCtx& c, const void* cells, double rc2, double* psi, double* partial) {
    launch_psi6_t<float>(c, cells, rc2, psi, partial);
}
unsigned psi6_blocks(const Geometry& g) {
    const dim3 grid = set_grid(g, dim3(kHistBX, kHistBY));
    return grid.x * grid.y * grid.z;
}
void launch_check_f32(const LaunchCtx& c, const void* cells, unsigned long long* out) {
    launch_check_t<float>(c, cells, out);
}

void launch_subsweep_f32_batch(const BatchCtx& c, void* arena, const SweepDraw* draws, int j, int k, bool track) {
    float* a = reinterpret_cast<float*>(arena);
#define HDMC_SUB_BATCH(ROWS, TRACK, DENSE, NSEL)                                                           \
    k_subsweep_f32_batch<ROWS, TRACK, DENSE, NSEL><<<c.sub_blocks, dim3(32, ROWS), 0, c.stream>>>(        \
        c.reps, c.sub_map, a, draws, c.R, j, k, c.partial, c.msd)
    // crowded cells in every replica: the dense kernel; one n_M shared by
    // every replica (4 or 8): the kernel with n_M fixed (the autotuner's
    // tracking launches keep the general one)
#define HDMC_SUB_BATCH_NSEL(ROWS, DENSE)                                                                   \
    do {                                                                                                   \
        if (c.nsel == 4) HDMC_SUB_BATCH(ROWS, false, DENSE, 4);                                            \
        else if (c.nsel == 8) HDMC_SUB_BATCH(ROWS, false, DENSE, 8);                                       \
        else HDMC_SUB_BATCH(ROWS, false, DENSE, 0);                                                        \
    } while (0)
#define HDMC_SUB_BATCH_ROWS(ROWS)                                                                          \
    do {                                                                                                   \
        if (track) HDMC_SUB_BATCH(ROWS, true, false, 0);                                                   \
        else if (c.dense) HDMC_SUB_BATCH_NSEL(ROWS, true);                                                 \
        else HDMC_SUB_BATCH_NSEL(ROWS, false);                                                             \
    } while (0)
    if (c.rows == 1) HDMC_SUB_BATCH_ROWS(1);
    else if (c.rows == 2) HDMC_SUB_BATCH_ROWS(2);
    else if (c.rows == 8) HDMC_SUB_BATCH_ROWS(8);
    else HDMC_SUB_BATCH_ROWS(4);
#undef HDMC_SUB_BATCH_ROWS
#undef HDMC_SUB_BATCH_NSEL
#undef HDMC_SUB_BATCH
}

void launch_shift_batch(const BatchCtx& c, int prec, const void* src, void* dst, const SweepDraw* draws, int j) {
    if (prec == 1)
        k_shift_batch<float><<<c.sh_blocks, dim3(kShiftBX, kShiftBY), 0, c.stream>>>(
            c.reps, c.sh_map, reinterpret_cast<const float*>(src), reinterpret_cast<float*>(dst), draws, c.R, j, c.sts);
    else
        k_shift_batch<double><<<c.sh_blocks, dim3(kShiftBX, kShiftBY), 0, c.stream>>>(
            c.reps, c.sh_map, reinterpret_cast<const double*>(src), reinterpret_cast<double*>(dst), draws, c.R, j,
            c.sts);
}

void launch_hist_batch(const BatchCtx& c, int prec, const void* arena) {
    if (prec == 1)
        k_hist_batch<float><<<c.hi_blocks, dim3(kHistBX, kHistBY), 0, c.stream>>>(
            c.reps, c.hi_map, reinterpret_cast<const float*>(arena), c.edges2, c.hist);
    else
        k_hist_batch<double><<<c.hi_blocks, dim3(kHistBX, kHistBY), 0, c.stream>>>(
            c.reps, c.hi_map, reinterpret_cast<const double*>(arena), c.edges2, c.hist);
}
}  // namespace hdmc
