// hdmc_batch.cu -- batched replicas: many independent hard-disk systems of
// different size and density advanced together, each pipeline stage one
// launch over all replicas, recorded into CUDA graphs.
//
// Each replica is exactly the system hdmc_create would build from the same
// arguments (same start, same random streams), so a replica's trajectory is
// bit-identical to the single-system run; batching only changes how the work
// is laid out on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "hdmc.h"
#include "hdmc_device.cuh"
#include "hdmc_host.h"

using namespace hdmc;

namespace {

constexpr int kChunk = 64;       // sweeps per recorded graph
constexpr size_t kAlign = 256;
constexpr int kRowsChoices[4] = {1, 2, 4, 8};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int ceil_div(int a, int b) { return (a + b - 1) / b; }

struct BatchLayout {
    size_t arena, table, states, partial, hist, edges, msd, reps, sub_map, sh_map, hi_map, total;
    long long cells;        // cells over all replicas
    int max_sub_blocks;     // sub-sweep blocks at the smallest block height
    int sh_blocks, hi_blocks;
};

int sub_blocks_of(const Geometry& g, int rows) { return ceil_div(g.hx, 32) * ceil_div(g.hy, rows); }

BatchLayout batch_layout(const std::vector<SysDesc>& sys, int prec) {
    BatchLayout L{};
    const size_t el = prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    long long cells = 0;
    int maxsub = 0, sh = 0, hi = 0;
    for (const SysDesc& d : sys) {
        cells += d.g.C;
        maxsub += sub_blocks_of(d.g, 1);
        sh += ceil_div(d.g.hx, kShiftBX) * ceil_div(d.g.hy, kShiftBY) * 4;
        hi += ceil_div(d.g.hx, kHistBX) * ceil_div(d.g.hy, kHistBY) * 4;
    }
    const int R = (int)sys.size();
    L.cells = cells;
    L.max_sub_blocks = maxsub;
    L.sh_blocks = sh;
    L.hi_blocks = hi;
    L.arena = align_up((size_t)cells * 8 * el);
    L.table = align_up(sizeof(SweepDraw) * kChunk * (size_t)R);
    L.states = align_up(sizeof(DevState) * (size_t)R);
    L.partial = align_up(sizeof(unsigned long long) * 4 * (size_t)maxsub);
    L.hist = align_up(sizeof(unsigned long long) * kHistBins * (size_t)R);
    L.edges = align_up(sizeof(double) * (kHistBins + 1));
    L.msd = align_up(sizeof(double) * (size_t)R);
    L.reps = align_up(sizeof(ReplicaDesc) * (size_t)R);
    L.sub_map = align_up(sizeof(unsigned short) * (size_t)maxsub);
    L.sh_map = align_up(sizeof(unsigned short) * (size_t)sh);
    L.hi_map = align_up(sizeof(unsigned short) * (size_t)hi);
    L.total = 2 * L.arena + L.table + L.states + L.partial + L.hist + L.edges + L.msd + L.reps + L.sub_map +
              L.sh_map + L.hi_map;
    return L;
}

}  // namespace

struct hdmc_batch_handle {
    int R = 0;
    int prec = HDMC_FP32_LOCAL;
    std::vector<SysDesc> sys;
    std::vector<long long> cell_off;
    BatchLayout lay{};
    int rows = 4;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    char* ws = nullptr;
    bool own_ws = false;
    void* arena[2] = {nullptr, nullptr};
    int cur = 0;
    SweepDraw* table = nullptr;
    DevState* sts = nullptr;
    unsigned long long* partial = nullptr;
    unsigned long long* hist = nullptr;
    double* edges2 = nullptr;
    double* msd = nullptr;
    ReplicaDesc* reps = nullptr;
    unsigned short* sub_map = nullptr;
    unsigned short* sh_map = nullptr;
    unsigned short* hi_map = nullptr;
    int sub_blocks = 0;
    std::vector<ReplicaDesc> host_reps;
    std::vector<unsigned long long> counter_base;   // R x 4, folded from earlier block layouts
    uint64_t sweeps = 0;
    int64_t n_samples = 0;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;   // (sweeps, parity, rows)

    BatchCtx ctx(cudaStream_t s) const {
        BatchCtx c;
        c.stream = s;
        c.reps = reps;
        c.sub_map = sub_map;
        c.sh_map = sh_map;
        c.hi_map = hi_map;
        c.sub_blocks = sub_blocks;
        c.sh_blocks = lay.sh_blocks;
        c.hi_blocks = lay.hi_blocks;
        c.R = R;
        c.rows = rows;
        c.dense = true;
        for (const SysDesc& d : sys) c.dense = c.dense && d.g.dense;
        c.nsel = sys.empty() ? 0 : sys[0].g.nsel;
        for (const SysDesc& d : sys) c.nsel = d.g.nsel == c.nsel ? c.nsel : 0;
        c.sts = sts;
        c.partial = partial;
        c.hist = hist;
        c.edges2 = edges2;
        c.msd = msd;
        return c;
    }
    void drop_graphs() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }
};

namespace {

// Replica descriptors and block maps for sub-sweep block height `rows`.
int upload_layout(hdmc_batch_t* b, int rows) {
    const int R = b->R;
    std::vector<ReplicaDesc> reps(R);
    std::vector<unsigned short> sub, sh, hi;
    int sub0 = 0, sh0 = 0, hi0 = 0;
    for (int r = 0; r < R; ++r) {
        const Geometry& g = b->sys[r].g;
        ReplicaDesc& d = reps[r];
        d.g = g;
        d.g.check = &b->sts[r].error;
        d.cell_off = b->cell_off[r];
        d.sub_gx = ceil_div(g.hx, 32);
        d.sub_block0 = sub0;
        d.part_off = sub0;
        const int ns = sub_blocks_of(g, rows);
        sub.insert(sub.end(), ns, (unsigned short)r);
        sub0 += ns;
        d.sh_gx = ceil_div(g.hx, kShiftBX);
        d.sh_gy = ceil_div(g.hy, kShiftBY);
        d.sh_block0 = sh0;
        const int nsh = d.sh_gx * d.sh_gy * 4;
        sh.insert(sh.end(), nsh, (unsigned short)r);
        sh0 += nsh;
        d.hi_gx = ceil_div(g.hx, kHistBX);
        d.hi_gy = ceil_div(g.hy, kHistBY);
        d.hi_block0 = hi0;
        const int nhi = d.hi_gx * d.hi_gy * 4;
        hi.insert(hi.end(), nhi, (unsigned short)r);
        hi0 += nhi;
    }
    // kernels already enqueued on the batch's stream read the old descriptors
    int e = cuda_code(cudaStreamSynchronize(b->stream));
    if (!e) e = cuda_code(cudaMemcpy(b->reps, reps.data(), sizeof(ReplicaDesc) * R, cudaMemcpyHostToDevice));
    if (!e) e = cuda_code(cudaMemcpy(b->sub_map, sub.data(), sizeof(unsigned short) * sub.size(), cudaMemcpyHostToDevice));
    if (!e) e = cuda_code(cudaMemcpy(b->sh_map, sh.data(), sizeof(unsigned short) * sh.size(), cudaMemcpyHostToDevice));
    if (!e) e = cuda_code(cudaMemcpy(b->hi_map, hi.data(), sizeof(unsigned short) * hi.size(), cudaMemcpyHostToDevice));
    // the copies ran on the legacy default stream: finish them before work is
    // enqueued on the batch's stream, which need not wait for it
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    if (e) return e;
    b->host_reps = reps;
    b->sub_blocks = sub0;
    b->rows = rows;
    return HDMC_OK;
}

// Per-replica counters of the current block layout, plus the folded base.
int read_counters(hdmc_batch_t* b, std::vector<unsigned long long>& out) {
    int e = cuda_code(cudaStreamSynchronize(b->stream));
    if (e) return e;
    std::vector<unsigned long long> part(4 * (size_t)b->sub_blocks);
    e = cuda_code(cudaMemcpy(part.data(), b->partial, sizeof(unsigned long long) * part.size(),
                             cudaMemcpyDeviceToHost));
    if (e) return e;
    out = b->counter_base;
    for (int r = 0; r < b->R; ++r) {
        const ReplicaDesc& d = b->host_reps[r];
        const int ns = sub_blocks_of(d.g, b->rows);
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < 4; ++k) out[4 * r + k] += part[4 * (size_t)(d.part_off + i) + k];
    }
    return HDMC_OK;
}

// Changes the sub-sweep block height, folding the counters of the old layout.
int set_rows(hdmc_batch_t* b, int rows) {
    if (rows == b->rows) return HDMC_OK;
    std::vector<unsigned long long> tot;
    int e = read_counters(b, tot);
    if (e) return e;
    b->counter_base = tot;
    e = cuda_code(cudaMemset(b->partial, 0, b->lay.partial));
    if (!e) e = upload_layout(b, rows);
    return e;
}

void enqueue_batch_sweeps(hdmc_batch_t* b, cudaStream_t s, int K, int parity, bool track) {
    const BatchCtx c = b->ctx(s);
    launch_draws_batch(s, b->reps, b->sts, b->table, b->R, K);
    for (int j = 0; j < K; ++j) {
        void* a = b->arena[parity ^ (j & 1)];
        void* o = b->arena[parity ^ (j & 1) ^ 1];
        for (int k = 0; k < 4; ++k) {
            if (b->prec == HDMC_FP64) launch_subsweep_f64_batch(c, a, b->table, j, k);
            else launch_subsweep_f32_batch(c, a, b->table, j, k, track);
        }
        launch_shift_batch(c, b->prec, a, o, b->table, j);
    }
}

int batch_graph(hdmc_batch_t* b, int K, cudaGraphExec_t& exec) {
    const auto key = std::make_tuple(K, b->cur, b->rows);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        exec = it->second;
        return HDMC_OK;
    }
    if (b->graphs.size() >= 12) b->drop_graphs();
    cudaGraph_t graph = nullptr;
    int e = cuda_code(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    if (e) return e;
    enqueue_batch_sweeps(b, b->cap, K, b->cur, false);
    e = cuda_code(cudaStreamEndCapture(b->cap, &graph));
    if (e) return e;
    e = cuda_code(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    if (e) return e;
    b->graphs[key] = exec;
    return HDMC_OK;
}

int check_batch(hdmc_batch_t* b) {
    int e = cuda_code(cudaStreamSynchronize(b->stream));
    if (e) return e;
    std::vector<DevState> st(b->R);
    e = cuda_code(cudaMemcpy(st.data(), b->sts, sizeof(DevState) * b->R, cudaMemcpyDeviceToHost));
    if (e) return e;
    for (const DevState& s : st)
        if (s.error) return error_code(s.error);
    return HDMC_OK;
}

}  // namespace

extern "C" {

size_t hdmc_batch_workspace_bytes(int R, const int64_t* N, const double* Lx, const double* Ly, double sigma,
                                  int precision) {
    if (R < 1 || R > 65535 || !N || !Lx || !Ly) return 0;
    if ((precision & 0xFF) != HDMC_FP64 && (precision & 0xFF) != HDMC_FP32_LOCAL) return 0;
    std::vector<SysDesc> sys(R);
    for (int r = 0; r < R; ++r)
        if (make_system(sys[r], N[r], Lx[r], Ly[r], sigma, 0.25, 4, 0, precision)) return 0;
    return batch_layout(sys, precision & 0xFF).total;
}

int hdmc_batch_create(hdmc_batch_t** out, int R, const int64_t* N, const double* Lx, const double* Ly,
                      double sigma, const double* d, const int32_t* nselect, const uint64_t* seeds, int precision,
                      void* dev_workspace, size_t workspace_bytes, void* stream) {
    if (!out) return HDMC_EINVAL;
    *out = nullptr;
    if (R < 1 || R > 65535 || !N || !Lx || !Ly || !d || !seeds) return HDMC_EINVAL;
    if (dev_workspace && ((uintptr_t)dev_workspace % kAlign)) return HDMC_EINVAL;
    std::vector<SysDesc> sys(R);
    for (int r = 0; r < R; ++r) {
        if (N[r] < 2 || (N[r] & 1)) return HDMC_EINVAL;
        const int e = make_system(sys[r], N[r], Lx[r], Ly[r], sigma, d[r], nselect ? nselect[r] : 4, seeds[r],
                                  precision);
        if (e) return e;
    }
    hdmc_batch_t* b = new (std::nothrow) hdmc_batch_t();
    if (!b) return HDMC_ENOMEM;
    b->R = R;
    b->prec = sys[0].prec;   // the bare precision (without the cell rule)
    b->sys = sys;
    b->stream = (cudaStream_t)stream;
    b->lay = batch_layout(sys, b->prec);
    b->counter_base.assign(4 * (size_t)R, 0);
    long long off = 0;
    for (int r = 0; r < R; ++r) {
        b->cell_off.push_back(off);
        off += sys[r].g.C;
    }
    int e = HDMC_OK;
    if (dev_workspace) {
        if (workspace_bytes < b->lay.total) e = HDMC_ENOMEM;
        b->ws = (char*)dev_workspace;
    } else {
        e = cuda_code(cudaMalloc((void**)&b->ws, b->lay.total));
        b->own_ws = e == HDMC_OK;
    }
    if (!e) e = cuda_code(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    if (e) {
        hdmc_batch_destroy(b);
        return e;
    }
    char* p = b->ws;
    b->arena[0] = p;
    p += b->lay.arena;
    b->arena[1] = p;
    p += b->lay.arena;
    b->table = (SweepDraw*)p;
    p += b->lay.table;
    b->sts = (DevState*)p;
    p += b->lay.states;
    b->partial = (unsigned long long*)p;
    p += b->lay.partial;
    b->hist = (unsigned long long*)p;
    p += b->lay.hist;
    b->edges2 = (double*)p;
    p += b->lay.edges;
    b->msd = (double*)p;
    p += b->lay.msd;
    b->reps = (ReplicaDesc*)p;
    p += b->lay.reps;
    b->sub_map = (unsigned short*)p;
    p += b->lay.sub_map;
    b->sh_map = (unsigned short*)p;
    p += b->lay.sh_map;
    b->hi_map = (unsigned short*)p;

    e = cuda_code(cudaMemset(b->ws + 2 * b->lay.arena, 0, b->lay.total - 2 * b->lay.arena));
    if (!e) {
        double E[kHistBins + 1];
        squared_edges(sigma, E);
        e = cuda_code(cudaMemcpy(b->edges2, E, sizeof(E), cudaMemcpyHostToDevice));
    }
    if (!e) e = upload_layout(b, 4);
    for (int r = 0; r < R && !e; ++r) {
        HostState hs;
        e = start_state(sys[r], hs);
        std::vector<char> raw;
        if (!e) pack(sys[r], hs, raw);
        if (!e)
            e = cuda_code(cudaMemcpy((char*)b->arena[0] + (size_t)b->cell_off[r] * 8 * sys[r].coord_bytes(),
                                     raw.data(), raw.size(), cudaMemcpyHostToDevice));
    }
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    if (e) {
        hdmc_batch_destroy(b);
        return e;
    }
    *out = b;
    return HDMC_OK;
}

int hdmc_batch_sweep(hdmc_batch_t* b, int64_t n) {
    if (!b || n < 0) return HDMC_EINVAL;
    while (n > 0) {
        const int K = (int)std::min<int64_t>(n, kChunk);
        cudaGraphExec_t exec;
        int e = batch_graph(b, K, exec);
        if (e) return e;
        e = cuda_code(cudaGraphLaunch(exec, b->stream));
        if (e) return e;
        b->cur ^= K & 1;
        b->sweeps += (uint64_t)K;
        n -= K;
    }
    return HDMC_OK;
}

int hdmc_batch_sample(hdmc_batch_t* b) {
    if (!b) return HDMC_EINVAL;
    launch_hist_batch(b->ctx(b->stream), b->prec, b->arena[b->cur]);
    b->n_samples += 1;
    return cuda_code(cudaGetLastError());
}

int hdmc_batch_pressure(hdmc_batch_t* b, double* betaP_over_rho, double* g_contact, uint64_t* hist,
                        int64_t* n_samples) {
    if (!b) return HDMC_EINVAL;
    int e = HDMC_OK;
    if (b->n_samples == 0) e = hdmc_batch_sample(b);
    if (!e) e = check_batch(b);
    if (e) return e;
    std::vector<unsigned long long> hh((size_t)kHistBins * b->R);
    e = cuda_code(cudaMemcpy(hh.data(), b->hist, sizeof(unsigned long long) * hh.size(), cudaMemcpyDeviceToHost));
    if (!e) e = cuda_code(cudaMemsetAsync(b->hist, 0, sizeof(unsigned long long) * hh.size(), b->stream));
    if (e) return e;
    const int64_t ns = b->n_samples;
    b->n_samples = 0;
    for (int r = 0; r < b->R; ++r) {
        double g0;
        const double bp = pressure_from_hist(b->sys[r], hh.data() + (size_t)r * kHistBins, ns, &g0);
        if (betaP_over_rho) betaP_over_rho[r] = bp;
        if (g_contact) g_contact[r] = g0;
    }
    if (hist)
        for (size_t i = 0; i < hh.size(); ++i) hist[i] = hh[i];
    if (n_samples) *n_samples = ns;
    return HDMC_OK;
}

int hdmc_batch_get_state(hdmc_batch_t* b, int r, double* local, uint8_t* counts) {
    if (!b || r < 0 || r >= b->R) return HDMC_EINVAL;
    int e = check_batch(b);
    if (e) return e;
    const SysDesc& d = b->sys[r];
    std::vector<char> raw(d.cells_bytes());
    e = cuda_code(cudaMemcpy(raw.data(), (const char*)b->arena[b->cur] + (size_t)b->cell_off[r] * 8 * d.coord_bytes(),
                             raw.size(), cudaMemcpyDeviceToHost));
    if (e) return e;
    HostState hs;
    unpack(d, raw, hs);
    if (local) std::memcpy(local, hs.loc.data(), sizeof(double) * hs.loc.size());
    if (counts) std::memcpy(counts, hs.cnt.data(), hs.cnt.size());
    return HDMC_OK;
}

int hdmc_batch_set_state(hdmc_batch_t* b, int r, const double* local, const uint8_t* counts,
                         const double origin[2], uint64_t sweeps_done) {
    if (!b || r < 0 || r >= b->R || !local || !counts || !origin) return HDMC_EINVAL;
    const SysDesc& d = b->sys[r];
    HostState hs;
    int e = state_from_local(d, local, counts, hs);
    if (e) return e;
    std::vector<char> raw;
    pack(d, hs, raw);
    e = cuda_code(cudaStreamSynchronize(b->stream));
    if (!e)
        e = cuda_code(cudaMemcpy((char*)b->arena[b->cur] + (size_t)b->cell_off[r] * 8 * d.coord_bytes(), raw.data(),
                                 raw.size(), cudaMemcpyHostToDevice));
    DevState ds;
    if (!e) e = cuda_code(cudaMemcpy(&ds, b->sts + r, sizeof(ds), cudaMemcpyDeviceToHost));
    if (e) return e;
    ds.origin[0] = origin[0];
    ds.origin[1] = origin[1];
    ds.sweep_next = sweeps_done;
    ds.error = 0;
    e = cuda_code(cudaMemcpy(b->sts + r, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    return e;
}

int hdmc_batch_counters(hdmc_batch_t* b, uint64_t* out) {
    if (!b || !out) return HDMC_EINVAL;
    std::vector<unsigned long long> tot;
    int e = read_counters(b, tot);
    if (e) return e;
    for (size_t i = 0; i < tot.size(); ++i) out[i] = tot[i];
    return check_batch(b);
}

int hdmc_batch_info(hdmc_batch_t* b, int r, int32_t* mx, int32_t* my, double* wx, double* wy,
                    uint64_t* sweeps_done, double origin[2]) {
    if (!b || r < 0 || r >= b->R) return HDMC_EINVAL;
    const Geometry& g = b->sys[r].g;
    if (mx) *mx = g.mx;
    if (my) *my = g.my;
    if (wx) *wx = g.wx;
    if (wy) *wy = g.wy;
    if (sweeps_done) *sweeps_done = b->sweeps;
    if (origin) {
        int e = cuda_code(cudaStreamSynchronize(b->stream));
        DevState st;
        if (!e) e = cuda_code(cudaMemcpy(&st, b->sts + r, sizeof(st), cudaMemcpyDeviceToHost));
        if (e) return e;
        origin[0] = st.origin[0];
        origin[1] = st.origin[1];
    }
    return HDMC_OK;
}

int hdmc_batch_set_nselect(hdmc_batch_t* b, const int32_t* nselect) {
    if (!b || !nselect) return HDMC_EINVAL;
    for (int r = 0; r < b->R; ++r)
        if (nselect[r] < 1 || nselect[r] > 255) return HDMC_EINVAL;
    int e = cuda_code(cudaStreamSynchronize(b->stream));
    if (e) return e;
    for (int r = 0; r < b->R; ++r) b->sys[r].g.nsel = nselect[r];
    b->drop_graphs();   // the sub-sweep kernel depends on whether all replicas share one n_M
    return upload_layout(b, b->rows);
}

int hdmc_batch_set_balance(hdmc_batch_t* b, const int32_t* shuffle_particles, const int32_t* shuffle_sets) {
    if (!b || !shuffle_particles || !shuffle_sets) return HDMC_EINVAL;
    int e = cuda_code(cudaStreamSynchronize(b->stream));
    if (e) return e;
    for (int r = 0; r < b->R; ++r)
        b->sys[r].g.flags = (shuffle_particles[r] ? 0u : kNoParticleShuffle) | (shuffle_sets[r] ? 0u : kNoSetShuffle);
    return upload_layout(b, b->rows);   // descriptors are read at run time: recorded graphs stay valid
}

int hdmc_batch_set_rows(hdmc_batch_t* b, int32_t rows_per_block) {
    if (!b || (rows_per_block != 1 && rows_per_block != 2 && rows_per_block != 4 && rows_per_block != 8))
        return HDMC_EINVAL;
    if (b->prec != HDMC_FP32_LOCAL && rows_per_block != 4) return HDMC_EINVAL;
    return set_rows(b, rows_per_block);
}

int hdmc_batch_config(hdmc_batch_t* b, int32_t* rows_per_block, int32_t* nselect) {
    if (!b) return HDMC_EINVAL;
    if (rows_per_block) *rows_per_block = b->rows;
    if (nselect)
        for (int r = 0; r < b->R; ++r) nselect[r] = b->sys[r].g.nsel;
    return HDMC_OK;
}

int hdmc_batch_autotune(hdmc_batch_t* b, int64_t sweeps, int32_t* rows_per_block, int32_t* nselect_chosen) {
    if (!b || sweeps < 1 || sweeps > 4096) return HDMC_EINVAL;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HDMC_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HDMC_ECUDA;
    }
    int e = HDMC_OK;
    auto timed_sweeps = [&](float& ms) {
        cudaEventRecord(e0, b->stream);
        e = hdmc_batch_sweep(b, sweeps);
        cudaEventRecord(e1, b->stream);
        if (!e) e = cuda_code(cudaEventSynchronize(e1));
        if (!e) e = cuda_code(cudaEventElapsedTime(&ms, e0, e1));
    };
    // 1. block height of the binary32 sub-sweep: fastest recorded sweeps
    int best_rows = b->rows;
    if (b->prec == HDMC_FP32_LOCAL) {
        float best = 0.f;
        for (int rows : kRowsChoices) {
            if (!e) e = set_rows(b, rows);
            if (!e) e = hdmc_batch_sweep(b, std::min<int64_t>(sweeps, kChunk));   // record the graph, warm up
            float ms = 0.f;
            if (!e) timed_sweeps(ms);
            if (!e && (best == 0.f || ms < best)) {
                best = ms;
                best_rows = rows;
            }
        }
        if (!e) e = set_rows(b, best_rows);
    }
    // 2. n_M: largest net squared displacement per disk and second, summed
    // over the replicas (each disk's displacement over its cell updates, so
    // confinement by the cell walls counts against large n_M)
    int best_nsel = b->sys[0].g.nsel;
    if (!e && b->prec == HDMC_FP32_LOCAL) {
        double best = -1.0;
        const int choices[4] = {1, 2, 4, 8};
        std::vector<int32_t> ns(b->R);
        for (int nm : choices) {
            std::fill(ns.begin(), ns.end(), nm);
            if (!e) e = hdmc_batch_set_nselect(b, ns.data());
            if (!e) e = cuda_code(cudaMemsetAsync(b->msd, 0, sizeof(double) * b->R, b->stream));
            float ms = 0.f;
            if (!e) {
                cudaEventRecord(e0, b->stream);
                for (int64_t done = 0; done < sweeps && !e; done += kChunk) {
                    const int K = (int)std::min<int64_t>(sweeps - done, kChunk);
                    enqueue_batch_sweeps(b, b->stream, K, b->cur, true);
                    b->cur ^= K & 1;
                    b->sweeps += (uint64_t)K;
                    e = cuda_code(cudaGetLastError());
                }
                cudaEventRecord(e1, b->stream);
                if (!e) e = cuda_code(cudaEventSynchronize(e1));
                if (!e) e = cuda_code(cudaEventElapsedTime(&ms, e0, e1));
            }
            std::vector<double> msd(b->R);
            if (!e) e = cuda_code(cudaMemcpy(msd.data(), b->msd, sizeof(double) * b->R, cudaMemcpyDeviceToHost));
            if (!e) {
                double rate = 0.0;
                for (int r = 0; r < b->R; ++r) rate += msd[r] / (double)b->sys[r].N;
                rate /= (double)ms;
                if (rate > best) {
                    best = rate;
                    best_nsel = nm;
                }
            }
        }
        std::fill(ns.begin(), ns.end(), best_nsel);
        if (!e) e = hdmc_batch_set_nselect(b, ns.data());
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return e;
    if (rows_per_block) *rows_per_block = b->rows;
    if (nselect_chosen) *nselect_chosen = best_nsel;
    return check_batch(b);
}

int hdmc_batch_psi6(hdmc_batch_t* b, double r_cut, double* out) {
    if (!b || !out || !(r_cut > 0.0)) return HDMC_EINVAL;
    for (int r = 0; r < b->R; ++r) {
        const Geometry& g = b->sys[r].g;
        const double wmin = b->prec == HDMC_FP64 ? std::min(g.wx, g.wy) : std::min((double)g.wxf, (double)g.wyf);
        if (!(r_cut <= 2.0 * wmin)) return HDMC_EINVAL;
    }
    // one launch per replica on its slice of the arena; block sums in the
    // idle half of the double buffer (scratch between sweeps)
    const cudaStream_t s = b->stream;
    const size_t el = b->prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    std::vector<size_t> off(b->R + 1, 0);
    for (int r = 0; r < b->R; ++r) off[r + 1] = off[r] + 4 * (size_t)psi6_blocks(b->sys[r].g);
    if (sizeof(double) * off[b->R] > b->lay.arena) return HDMC_EINVAL;
    double* partial = reinterpret_cast<double*>(b->arena[b->cur ^ 1]);
    const char* cur = static_cast<const char*>(b->arena[b->cur]);
    int e = HDMC_OK;
    for (int r = 0; r < b->R && !e; ++r) {
        LaunchCtx c;
        c.g = b->sys[r].g;
        c.stream = s;
        const void* cells = cur + (size_t)b->cell_off[r] * 8 * el;
        if (b->prec == HDMC_FP64) launch_psi6_f64(c, cells, r_cut * r_cut, nullptr, partial + off[r]);
        else launch_psi6_f32(c, cells, r_cut * r_cut, nullptr, partial + off[r]);
        e = cuda_code(cudaGetLastError());
    }
    std::vector<double> part(off[b->R]);
    if (!e)
        e = cuda_code(cudaMemcpyAsync(part.data(), partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    for (int r = 0; r < b->R; ++r) {
        double sum[4] = {0, 0, 0, 0};
        for (size_t i = off[r]; i < off[r + 1]; i += 4)
            for (int k = 0; k < 4; ++k) sum[k] += part[i + k];
        for (int k = 0; k < 4; ++k) out[4 * r + k] = sum[k] / (double)b->sys[r].N;
    }
    return HDMC_OK;
}

// ---- batch snapshots ------------------------------------------------------------------
namespace {

constexpr char kBatchMagic[8] = {'H', 'D', 'M', 'C', 'B', 'S', 'N', '1'};
constexpr uint32_t kBatchVersion = 1;
constexpr size_t kBatchHeader = 256;

struct BatchSnapHeader {
    char magic[8];
    uint32_t version, precision;
    int32_t R, rows;
    uint64_t sweeps;
    int64_t n_samples;
    uint64_t off_reps, off_states, off_counters, off_hist, off_cells, cell_bytes, total;
};
static_assert(sizeof(BatchSnapHeader) <= kBatchHeader, "batch snapshot header");

struct BatchSnapReplica {
    int64_t N;
    double Lx, Ly, sigma, d;
    int32_t nsel, mx, my, pad0;
    uint32_t key0, key1, flags, pad1;
};

struct BatchSnapLayout {
    size_t reps, states, counters, hist, cells, cell_bytes, total;
};

BatchSnapLayout batch_snap_layout(const hdmc_batch_t* b) {
    BatchSnapLayout L;
    size_t p = kBatchHeader;
    L.reps = p;
    p += align_up(sizeof(BatchSnapReplica) * (size_t)b->R);
    L.states = p;
    p += align_up(sizeof(DevState) * (size_t)b->R);
    L.counters = p;
    p += align_up(sizeof(unsigned long long) * 4 * (size_t)b->R);
    L.hist = p;
    p += align_up(sizeof(unsigned long long) * kHistBins * (size_t)b->R);
    L.cells = p;
    L.cell_bytes = (size_t)b->lay.cells * 8 * (b->prec == HDMC_FP64 ? sizeof(double) : sizeof(float));
    L.total = p + L.cell_bytes;
    return L;
}

}  // namespace

size_t hdmc_batch_snapshot_bytes(const hdmc_batch_t* b) { return b ? batch_snap_layout(b).total : 0; }

int hdmc_batch_save(hdmc_batch_t* b, void* buf, size_t bytes) {
    if (!b || !buf) return HDMC_EINVAL;
    const BatchSnapLayout L = batch_snap_layout(b);
    if (bytes < L.total) return HDMC_EINVAL;
    char* p = static_cast<char*>(buf);
    std::vector<unsigned long long> tot;
    int e = read_counters(b, tot);   // synchronises
    if (e) return e;
    std::memset(p, 0, L.cells);
    BatchSnapHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kBatchMagic, sizeof(kBatchMagic));
    hd.version = kBatchVersion;
    hd.precision = (uint32_t)b->prec;
    hd.R = b->R;
    hd.rows = b->rows;
    hd.sweeps = b->sweeps;
    hd.n_samples = b->n_samples;
    hd.off_reps = L.reps;
    hd.off_states = L.states;
    hd.off_counters = L.counters;
    hd.off_hist = L.hist;
    hd.off_cells = L.cells;
    hd.cell_bytes = L.cell_bytes;
    hd.total = L.total;
    std::memcpy(p, &hd, sizeof(hd));
    for (int r = 0; r < b->R; ++r) {
        const SysDesc& d = b->sys[r];
        BatchSnapReplica rec;
        std::memset(&rec, 0, sizeof(rec));
        rec.N = d.N;
        rec.Lx = d.Lx;
        rec.Ly = d.Ly;
        rec.sigma = d.g.sigma;
        rec.d = d.g.d;
        rec.nsel = d.g.nsel;
        rec.mx = d.g.mx;
        rec.my = d.g.my;
        rec.key0 = d.g.key0;
        rec.key1 = d.g.key1;
        rec.flags = d.g.flags;
        std::memcpy(p + L.reps + sizeof(rec) * (size_t)r, &rec, sizeof(rec));
    }
    std::memcpy(p + L.counters, tot.data(), sizeof(unsigned long long) * tot.size());
    const cudaStream_t s = b->stream;
    e = cuda_code(cudaMemcpyAsync(p + L.states, b->sts, sizeof(DevState) * (size_t)b->R, cudaMemcpyDeviceToHost, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(p + L.hist, b->hist, sizeof(unsigned long long) * kHistBins * (size_t)b->R,
                                      cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaMemcpyAsync(p + L.cells, b->arena[b->cur], L.cell_bytes, cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    for (int r = 0; r < b->R; ++r) {
        DevState ds;
        std::memcpy(&ds, p + L.states + sizeof(DevState) * (size_t)r, sizeof(ds));
        if (ds.error) return error_code(ds.error);
    }
    return HDMC_OK;
}

int hdmc_batch_load(hdmc_batch_t* b, const void* buf, size_t bytes) {
    if (!b || !buf) return HDMC_EINVAL;
    const BatchSnapLayout L = batch_snap_layout(b);
    if (bytes < L.total) return HDMC_EINVAL;
    const char* p = static_cast<const char*>(buf);
    BatchSnapHeader hd;
    std::memcpy(&hd, p, sizeof(hd));
    if (std::memcmp(hd.magic, kBatchMagic, sizeof(kBatchMagic)) != 0 || hd.version != kBatchVersion ||
        hd.precision != (uint32_t)b->prec || hd.R != b->R || hd.n_samples < 0 || hd.off_reps != L.reps ||
        hd.off_states != L.states || hd.off_counters != L.counters || hd.off_hist != L.hist ||
        hd.off_cells != L.cells || hd.cell_bytes != L.cell_bytes || hd.total != L.total)
        return HDMC_EINVAL;
    std::vector<BatchSnapReplica> recs(b->R);
    for (int r = 0; r < b->R; ++r) {
        BatchSnapReplica& rec = recs[r];
        std::memcpy(&rec, p + L.reps + sizeof(rec) * (size_t)r, sizeof(rec));
        const SysDesc& d = b->sys[r];
        if (rec.N != d.N || rec.Lx != d.Lx || rec.Ly != d.Ly || rec.sigma != d.g.sigma || rec.mx != d.g.mx ||
            rec.my != d.g.my || rec.nsel < 1 || rec.nsel > 255 || !(rec.d > 0) || !(rec.d < 0.5 * d.g.wx) ||
            !(rec.d < 0.5 * d.g.wy) || (rec.flags & ~(kNoParticleShuffle | kNoSetShuffle)) != 0)
            return HDMC_EINVAL;
        DevState ds;
        std::memcpy(&ds, p + L.states + sizeof(DevState) * (size_t)r, sizeof(ds));
        if (ds.error != 0 || !std::isfinite(ds.origin[0]) || !std::isfinite(ds.origin[1])) return HDMC_EINVAL;
    }
    // cells into the idle half of the double buffer, checked there replica by
    // replica (results in the draw table, scratch until the next sweep)
    const cudaStream_t s = b->stream;
    const size_t el = b->prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    char* idle = static_cast<char*>(b->arena[b->cur ^ 1]);
    unsigned long long* res = reinterpret_cast<unsigned long long*>(b->table);
    int e = cuda_code(cudaStreamSynchronize(s));
    if (!e) e = cuda_code(cudaMemsetAsync(res, 0, sizeof(unsigned long long) * 2 * (size_t)b->R, s));
    if (!e) e = cuda_code(cudaMemcpyAsync(idle, p + L.cells, L.cell_bytes, cudaMemcpyHostToDevice, s));
    for (int r = 0; r < b->R && !e; ++r) {
        LaunchCtx c;
        c.g = b->sys[r].g;
        c.stream = s;
        void* cells = idle + (size_t)b->cell_off[r] * 8 * el;
        if (b->prec == HDMC_FP64) launch_check_f64(c, cells, res + 2 * r);
        else launch_check_f32(c, cells, res + 2 * r);
        e = cuda_code(cudaGetLastError());
    }
    std::vector<unsigned long long> got(2 * (size_t)b->R);
    if (!e)
        e = cuda_code(cudaMemcpyAsync(got.data(), res, sizeof(unsigned long long) * got.size(), cudaMemcpyDeviceToHost,
                                      s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    for (int r = 0; r < b->R; ++r)
        if (got[2 * r + 1] != 0 || got[2 * r] != (unsigned long long)b->sys[r].N) return HDMC_EINVAL;
    // commit
    e = cuda_code(cudaMemcpyAsync(b->sts, p + L.states, sizeof(DevState) * (size_t)b->R, cudaMemcpyHostToDevice, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(b->hist, p + L.hist, sizeof(unsigned long long) * kHistBins * (size_t)b->R,
                                      cudaMemcpyHostToDevice, s));
    if (!e) e = cuda_code(cudaMemsetAsync(b->partial, 0, b->lay.partial, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    b->counter_base.assign(4 * (size_t)b->R, 0);
    std::memcpy(b->counter_base.data(), p + L.counters, sizeof(unsigned long long) * 4 * (size_t)b->R);
    for (int r = 0; r < b->R; ++r) {
        Geometry& g = b->sys[r].g;
        g.d = recs[r].d;
        g.df = (float)recs[r].d;
        g.nsel = recs[r].nsel;
        g.key0 = recs[r].key0;
        g.key1 = recs[r].key1;
        g.flags = recs[r].flags;
    }
    b->cur ^= 1;
    b->sweeps = hd.sweeps;
    b->n_samples = hd.n_samples;
    b->drop_graphs();
    const int rows = (b->prec == HDMC_FP32_LOCAL &&
                      (hd.rows == 1 || hd.rows == 2 || hd.rows == 4 || hd.rows == 8)) ? hd.rows : b->rows;
    return upload_layout(b, rows);
}

void hdmc_batch_destroy(hdmc_batch_t* b) {
    if (!b) return;
    if (b->stream || b->ws) cudaStreamSynchronize(b->stream);
    b->drop_graphs();
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_ws && b->ws) cudaFree(b->ws);
    delete b;
}

}  // extern "C"
