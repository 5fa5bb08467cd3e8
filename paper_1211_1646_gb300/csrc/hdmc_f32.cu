// Binary32 cell-local coordinates (HDMC_FP32_LOCAL).
#include "hdmc_kernels.cuh"

namespace hdmc {
void launch_subsweep_f32(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k) {
    k_subsweep_f32<<<subsweep_grid(c.g), dim3(32, 4), 0, c.stream>>>(c.g, reinterpret_cast<float*>(cells), draw, k,
                                                                     c.partial);
}
void launch_shift_f32(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw) {
    launch_shift_t<float>(c, src, dst, draw);
}
void launch_hist_f32(const LaunchCtx& c, const void* cells) { launch_hist_t<float>(c, cells); }
}  // namespace hdmc
