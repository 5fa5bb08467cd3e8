// Binary64 cell-local coordinates (HDMC_FP64).
#include "hdmc_kernels.cuh"

namespace hdmc {
void launch_subsweep_f64(const LaunchCtx& c, void* cells, const SweepDraw* draw, int k) {
    launch_on(c, k_subsweep_f64, dim3((unsigned)((c.g.hx + 31) / 32), (unsigned)c.g.hy), dim3(32, 1), c.g,
              reinterpret_cast<double*>(cells), draw, k, c.partial);
}
void launch_shift_f64(const LaunchCtx& c, const void* src, void* dst, const SweepDraw* draw) {
    launch_shift_t<double>(c, src, dst, draw);
}
void launch_hist_f64(const LaunchCtx& c, const void* cells) { launch_hist_t<double>(c, cells); }
void launch_psi6_f64(const LaunchCtx& c, const void* cells, double rc2, double* psi, double* partial) {
    launch_psi6_t<double>(c, cells, rc2, psi, partial);
}
void launch_check_f64(const LaunchCtx& c, const void* cells, unsigned long long* out) {
    launch_check_t<double>(c, cells, out);
}

void launch_subsweep_f64_batch(const BatchCtx& c, void* arena, const SweepDraw* draws, int j, int k) {
    k_subsweep_f64_batch<<<c.sub_blocks, dim3(32, 4), 0, c.stream>>>(c.reps, c.sub_map, reinterpret_cast<double*>(arena),
                                                                      draws, c.R, j, k, c.partial);
}
}  // namespace hdmc
