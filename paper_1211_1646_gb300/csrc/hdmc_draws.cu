// Sweep-level draws (Alg. 1: set order and grid shift) computed on the device, so that
// a recorded graph of many sweeps advances its own sweep counter.
#include "hdmc_device.cuh"

namespace hdmc {

// Single block: reads the next index, fills table[0..count), advances it.
__global__ void __launch_bounds__(256) k_draws(const Geometry g, SweepDraw* __restrict__ table, int count,
                                               DevState* __restrict__ st, int sweep_mode) {
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = sweep_mode ? st->sweep_next : st->shift_next;
    __syncthreads();
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
        const uint32_t index = (uint32_t)(base + (unsigned long long)j);
        table[j] = make_draw(g, index, sweep_mode ? kDomSweep : kDomShift, sweep_mode != 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sweep_mode) st->sweep_next = base + (unsigned long long)count;
        else st->shift_next = base + (unsigned long long)count;
    }
}

void launch_draws(const LaunchCtx& c, SweepDraw* table, int count, bool sweep_mode) {
    k_draws<<<1, 256, 0, c.stream>>>(c.g, table, count, c.st, sweep_mode ? 1 : 0);
}

// One block per replica: fills draws[j*R + r] for j < count and advances
// the replica's sweep counter.
__global__ void __launch_bounds__(64) k_draws_batch(const ReplicaDesc* __restrict__ reps, DevState* __restrict__ sts,
                                                    SweepDraw* __restrict__ table, int R, int count) {
    const int r = blockIdx.x;
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = sts[r].sweep_next;
    __syncthreads();
    const Geometry g = reps[r].g;
    for (int j = threadIdx.x; j < count; j += blockDim.x)
        table[(size_t)j * R + r] = make_draw(g, (uint32_t)(base + (unsigned long long)j), kDomSweep, true);
    __syncthreads();
    if (threadIdx.x == 0) sts[r].sweep_next = base + (unsigned long long)count;
}

void launch_draws_batch(cudaStream_t s, const ReplicaDesc* reps, DevState* sts, SweepDraw* table, int R, int count) {
    k_draws_batch<<<R, 64, 0, s>>>(reps, sts, table, R, count);
}

dim3 subsweep_grid(const Geometry& g) {
    return dim3((unsigned)((g.hx + 31) / 32), (unsigned)((g.hy + kCounterRows - 1) / kCounterRows));
}

}  // namespace hdmc
