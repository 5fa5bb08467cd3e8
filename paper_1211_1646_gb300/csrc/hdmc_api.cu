// hdmc_api.cu -- host side of libhdmc.so: the C ABI declared in hdmc.h.
//
// Responsibilities: validating parameters, laying out the device workspace,
// building the hexagonal start and binning disks into cells, recording
// sweeps into CUDA graphs (one graph node per kernel; the sweep index and the
// double-buffer parity are advanced on the device, so a recorded graph is
// replayed as is), and the Sec. 4 pressure fit on the 200-bin histogram.
// Host floating point is compiled without contraction (-ffp-contract=off) so
// that the start configuration is the same on every host architecture.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "hdmc.h"
#include "hdmc_device.cuh"
#include "hdmc_host.h"

using namespace hdmc;

namespace {

constexpr int kChunk = 64;       // sweeps per recorded graph
constexpr size_t kAlign = 256;   // workspace segment alignment

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t cells, table, shift_table, state, partial, hist, edges, check, total;
    int nblocks;
};

Layout make_layout(const Geometry& g, int prec) {
    Layout L;
    const size_t slot = prec == HDMC_FP64 ? sizeof(double2) : sizeof(float2);
    L.cells = align_up((size_t)g.C * kSlots * slot);
    L.table = align_up(sizeof(SweepDraw) * kChunk);
    L.shift_table = align_up(sizeof(SweepDraw));
    L.state = align_up(sizeof(DevState));
    const dim3 grid = subsweep_grid(g);
    L.nblocks = (int)(grid.x * grid.y);
    L.partial = align_up(sizeof(unsigned long long) * 4 * (size_t)L.nblocks);
    L.hist = align_up(sizeof(unsigned long long) * kHistBins);
    L.edges = align_up(sizeof(double) * (kHistBins + 1));
    L.check = align_up(2 * sizeof(unsigned long long));
    L.total = 2 * L.cells + L.table + L.shift_table + L.state + L.partial + L.hist + L.edges + L.check;
    return L;
}


}  // namespace

struct hdmc_handle {
    Geometry g;
    int64_t N;
    double Lx, Ly;
    int prec;
    cudaStream_t stream = nullptr;   // caller's stream (nullptr = legacy default stream)
    cudaStream_t cap = nullptr;      // private stream used only to record graphs
    char* ws = nullptr;
    bool own_ws = false;
    Layout lay;
    void* cells[2] = {nullptr, nullptr};
    int cur = 0;
    SweepDraw* table = nullptr;
    SweepDraw* shift_table = nullptr;
    DevState* st = nullptr;
    unsigned long long* partial = nullptr;
    unsigned long long* hist = nullptr;
    double* edges2 = nullptr;
    unsigned long long* check = nullptr;   // snapshot check: {disks, bad cell flag}
    uint64_t sweeps = 0, shifts = 0;
    int64_t n_samples = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (sweeps, parity) -> graph
    // strip of a decomposed system (Sec. 6); nstrips == 0 for a whole system
    int nstrips = 0, strip = 0;
    int r0 = 0, r1 = 0;       // global rows [r0, r1) owned by the strip
    int myg = 0;              // rows of the whole grid
    bool pending = false;     // sub-sweeps of a sweep done, its shift not yet

    LaunchCtx ctx(cudaStream_t s) const {
        LaunchCtx c;
        c.g = g;
        c.stream = s;
        c.st = st;
        c.partial = partial;
        c.hist = hist;
        c.edges2 = edges2;
        return c;
    }
    void drop_graphs() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }
    SysDesc desc() const {
        SysDesc d;
        d.g = g;
        d.N = N;
        d.Lx = Lx;
        d.Ly = Ly;
        d.prec = prec;
        return d;
    }
};

namespace {

int upload(hdmc_t* h, const HostState& hs) {
    std::vector<char> raw;
    pack(h->desc(), hs, raw);
    return cuda_code(cudaMemcpy(h->cells[h->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice));
}

int download(hdmc_t* h, HostState& hs) {
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    if (e) return e;
    std::vector<char> raw(h->lay.cells);
    e = cuda_code(cudaMemcpy(raw.data(), h->cells[h->cur], raw.size(), cudaMemcpyDeviceToHost));
    if (e) return e;
    unpack(h->desc(), raw, hs);
    return HDMC_OK;
}

int read_devstate(hdmc_t* h, DevState& ds) {
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    if (e) return e;
    return cuda_code(cudaMemcpy(&ds, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
}

int check_device(hdmc_t* h) {
    DevState ds;
    int e = read_devstate(h, ds);
    if (e) return e;
    return error_code(ds.error);
}

// ---- sweep driver ------------------------------------------------------------

// The draws kernel and the first sub-sweep after it are ordinary launches;
// every later kernel of the run is a programmatic dependent of the one
// before it (launch_on), so its blocks fill the SMs that the previous
// kernel's last blocks leave idle.
void enqueue_sweeps(hdmc_t* h, cudaStream_t s, int K, int parity) {
    LaunchCtx c = h->ctx(s);
    launch_draws(c, h->table, K, true);
    for (int j = 0; j < K; ++j) {
        void* a = h->cells[parity ^ (j & 1)];
        void* b = h->cells[parity ^ (j & 1) ^ 1];
        for (int k = 0; k < 4; ++k) {
            c.pdl = j > 0 || k > 0;
            if (h->prec == HDMC_FP64) launch_subsweep_f64(c, a, h->table + j, k);
            else launch_subsweep_f32(c, a, h->table + j, k);
        }
        if (h->prec == HDMC_FP64) launch_shift_f64(c, a, b, h->table + j);
        else launch_shift_f32(c, a, b, h->table + j);
    }
}

int sweep_graph(hdmc_t* h, int K, cudaGraphExec_t& exec) {
    const auto key = std::make_pair(K, h->cur);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        exec = it->second;
        return HDMC_OK;
    }
    if (h->graphs.size() >= 8) h->drop_graphs();
    cudaGraph_t graph = nullptr;
    int e = cuda_code(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    if (e) return e;
    enqueue_sweeps(h, h->cap, K, h->cur);
    e = cuda_code(cudaStreamEndCapture(h->cap, &graph));
    if (e) return e;
    e = cuda_code(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    if (e) return e;
    h->graphs[key] = exec;
    return HDMC_OK;
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================
extern "C" {

size_t hdmc_workspace_bytes(int64_t N, double Lx, double Ly, double sigma, int precision) {
    int mx, my;
    double wx, wy;
    const int rule = precision >> 8;
    precision &= 0xFF;
    if (N < 1 || (precision != HDMC_FP64 && precision != HDMC_FP32_LOCAL)) return 0;
    if (!make_grid(Lx, Ly, sigma, mx, my, wx, wy, rule)) return 0;
    if ((int64_t)mx * my >= (int64_t(1) << 32)) return 0;   // as hdmc_create
    Geometry g{};
    g.mx = mx;
    g.my = my;
    g.hx = mx / 2;
    g.hy = my / 2;
    g.cq = (long long)g.hx * g.hy;
    g.C = (long long)mx * my;
    return make_layout(g, precision).total;
}

int hdmc_create(hdmc_t** out, int64_t N, double Lx, double Ly, double sigma, double d, int nselect, uint64_t seed,
                int precision, void* dev_workspace, size_t workspace_bytes, void* stream) {
    if (!out) return HDMC_EINVAL;
    *out = nullptr;
    if (N < 2 || (N & 1)) return HDMC_EINVAL;
    SysDesc desc;
    int e0 = make_system(desc, N, Lx, Ly, sigma, d, nselect, seed, precision);
    if (e0) return e0;
    if (dev_workspace && ((uintptr_t)dev_workspace % kAlign)) return HDMC_EINVAL;

    hdmc_t* h = new (std::nothrow) hdmc_t();
    if (!h) return HDMC_ENOMEM;
    h->g = desc.g;
    h->N = N;
    h->Lx = Lx;
    h->Ly = Ly;
    h->prec = desc.prec;
    const Geometry& g = h->g;
    h->stream = (cudaStream_t)stream;
    h->lay = make_layout(g, desc.prec);

    int e = HDMC_OK;
    if (dev_workspace) {
        if (workspace_bytes < h->lay.total) e = HDMC_ENOMEM;
        h->ws = (char*)dev_workspace;
    } else {
        e = cuda_code(cudaMalloc((void**)&h->ws, h->lay.total));
        h->own_ws = e == HDMC_OK;
    }
    if (!e) e = cuda_code(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    if (e) {
        hdmc_destroy(h);
        return e;
    }
    char* p = h->ws;
    h->cells[0] = p;
    p += h->lay.cells;
    h->cells[1] = p;
    p += h->lay.cells;
    h->table = (SweepDraw*)p;
    p += h->lay.table;
    h->shift_table = (SweepDraw*)p;
    p += h->lay.shift_table;
    h->st = (DevState*)p;
    h->g.check = &h->st->error;
    p += h->lay.state;
    h->partial = (unsigned long long*)p;
    p += h->lay.partial;
    h->hist = (unsigned long long*)p;
    p += h->lay.hist;
    h->edges2 = (double*)p;
    p += h->lay.edges;
    h->check = (unsigned long long*)p;

    e = cuda_code(cudaMemset(h->ws + 2 * h->lay.cells, 0, h->lay.total - 2 * h->lay.cells));
    if (!e) {
        double E[kHistBins + 1];   // squared histogram bin edges (sigma + k dr)^2
        squared_edges(sigma, E);
        e = cuda_code(cudaMemcpy(h->edges2, E, sizeof(E), cudaMemcpyHostToDevice));
    }
    if (!e) {
        HostState hs;
        e = start_state(h->desc(), hs);
        if (!e) e = upload(h, hs);
    }
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    if (e) {
        hdmc_destroy(h);
        return e;
    }
    *out = h;
    return HDMC_OK;
}

int hdmc_set_positions(hdmc_t* h, const double* xy) {
    if (!h || !xy) return HDMC_EINVAL;
    if (h && h->nstrips) return HDMC_EINVAL;
    HostState hs;
    int e = bin_positions(h->desc(), xy, hs);
    if (e) return e;
    if (any_overlap(h->desc(), hs)) return HDMC_EOVERLAP;
    e = cuda_code(cudaStreamSynchronize(h->stream));
    if (!e) e = upload(h, hs);
    DevState ds;
    if (!e) e = read_devstate(h, ds);
    if (!e) {
        ds.origin[0] = ds.origin[1] = 0.0;
        e = cuda_code(cudaMemcpy(h->st, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    }
    // the copies ran on the legacy default stream: finish them before work is
    // enqueued on the handle's stream, which need not wait for it
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    return e;
}

int hdmc_sweep(hdmc_t* h, int64_t n) {
    if (!h || n < 0) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    while (n > 0) {
        const int K = (int)std::min<int64_t>(n, kChunk);
        cudaGraphExec_t exec;
        int e = sweep_graph(h, K, exec);
        if (e) return e;
        e = cuda_code(cudaGraphLaunch(exec, h->stream));
        if (e) return e;
        h->cur ^= K & 1;
        h->sweeps += (uint64_t)K;
        n -= K;
    }
    return HDMC_OK;
}

int hdmc_profile_sweeps(hdmc_t* h, int64_t n, double* ms_subsweep, double* ms_shift, double* ms_draws) {
    if (!h || n < 0) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    const int nev = 2;
    cudaEvent_t ev[nev];
    for (int i = 0; i < nev; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return HDMC_ECUDA;
        }
    const LaunchCtx c = h->ctx(h->stream);
    double t_sub = 0, t_shift = 0, t_draw = 0;
    int64_t n_sub = 0, n_shift = 0, n_draw = 0;
    int e = HDMC_OK;
    auto timed = [&](auto&& launch, double& acc, int64_t& cnt) {
        if (e) return;
        cudaEventRecord(ev[0], h->stream);
        launch();
        cudaEventRecord(ev[1], h->stream);
        e = cuda_code(cudaEventSynchronize(ev[1]));
        float ms = 0.f;
        if (!e) e = cuda_code(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        acc += ms;
        cnt += 1;
    };
    while (n > 0 && !e) {
        const int K = (int)std::min<int64_t>(n, kChunk);
        timed([&] { launch_draws(c, h->table, K, true); }, t_draw, n_draw);
        for (int j = 0; j < K && !e; ++j) {
            void* a = h->cells[h->cur];
            void* b = h->cells[h->cur ^ 1];
            for (int k = 0; k < 4; ++k)
                timed([&] {
                    if (h->prec == HDMC_FP64) launch_subsweep_f64(c, a, h->table + j, k);
                    else launch_subsweep_f32(c, a, h->table + j, k);
                }, t_sub, n_sub);
            timed([&] {
                if (h->prec == HDMC_FP64) launch_shift_f64(c, a, b, h->table + j);
                else launch_shift_f32(c, a, b, h->table + j);
            }, t_shift, n_shift);
            h->cur ^= 1;
            h->sweeps += 1;
        }
        n -= K;
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    if (e) return e;
    if (ms_subsweep) *ms_subsweep = n_sub ? t_sub / n_sub : 0.0;
    if (ms_shift) *ms_shift = n_shift ? t_shift / n_shift : 0.0;
    if (ms_draws) *ms_draws = n_draw ? t_draw / n_draw : 0.0;
    return check_device(h);
}

// stage 1: draws + the four sub-sweeps of each sweep, no shift (the cells stay
// in one buffer); stage 2: draws + the shift of each sweep.  Programmatic
// dependent launches as in enqueue_sweeps.
void enqueue_stage(hdmc_t* h, cudaStream_t s, int K, int parity, int stage) {
    LaunchCtx c = h->ctx(s);
    launch_draws(c, h->table, K, true);
    for (int j = 0; j < K; ++j) {
        if (stage == 1) {
            void* a = h->cells[parity];
            for (int k = 0; k < 4; ++k) {
                c.pdl = j > 0 || k > 0;
                if (h->prec == HDMC_FP64) launch_subsweep_f64(c, a, h->table + j, k);
                else launch_subsweep_f32(c, a, h->table + j, k);
            }
        } else {
            void* a = h->cells[parity ^ (j & 1)];
            void* b = h->cells[parity ^ (j & 1) ^ 1];
            c.pdl = j > 0;
            if (h->prec == HDMC_FP64) launch_shift_f64(c, a, b, h->table + j);
            else launch_shift_f32(c, a, b, h->table + j);
        }
    }
}

int hdmc_profile_stages(hdmc_t* h, int64_t n, double* ms_subsweep, double* ms_shift) {
    if (!h || n < 1) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return HDMC_ECUDA;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return HDMC_ECUDA;
    }
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    double per[3] = {0.0, 0.0, 0.0};
    for (int stage = 1; stage <= 2 && !e; ++stage) {
        const int K = (int)std::min<int64_t>(n, kChunk);
        const int64_t reps = (n + K - 1) / K;
        // one recorded graph per parity of the state buffer
        cudaGraphExec_t exec[2] = {nullptr, nullptr};
        for (int par = 0; par < 2 && !e; ++par) {
            if (stage == 1 && par == 1) break;
            cudaGraph_t graph = nullptr;
            e = cuda_code(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            if (e) break;
            enqueue_stage(h, h->cap, K, stage == 1 ? h->cur : (h->cur ^ par), stage);
            e = cuda_code(cudaStreamEndCapture(h->cap, &graph));
            if (!e) e = cuda_code(cudaGraphInstantiate(&exec[par], graph, 0));
            if (graph) cudaGraphDestroy(graph);
        }
        float ms = 0.f;
        if (!e) e = cuda_code(cudaEventRecord(ev[0], h->stream));
        int par = 0;
        for (int64_t r = 0; r < reps && !e; ++r) {
            e = cuda_code(cudaGraphLaunch(exec[stage == 1 ? 0 : par], h->stream));
            h->sweeps += (uint64_t)K;
            if (stage == 2) par ^= K & 1;
        }
        if (!e) e = cuda_code(cudaEventRecord(ev[1], h->stream));
        if (!e) e = cuda_code(cudaEventSynchronize(ev[1]));
        if (!e) e = cuda_code(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        if (stage == 2) h->cur ^= par;
        for (int q = 0; q < 2; ++q)
            if (exec[q]) cudaGraphExecDestroy(exec[q]);
        per[stage] = (double)ms / (double)(reps * K * (stage == 1 ? 4 : 1));
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e) return e;
    if (ms_subsweep) *ms_subsweep = per[1];
    if (ms_shift) *ms_shift = per[2];
    return check_device(h);
}

int hdmc_shift(hdmc_t* h) {
    if (!h) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    const LaunchCtx c = h->ctx(h->stream);
    launch_draws(c, h->shift_table, 1, false);
    if (h->prec == HDMC_FP64) launch_shift_f64(c, h->cells[h->cur], h->cells[h->cur ^ 1], h->shift_table);
    else launch_shift_f32(c, h->cells[h->cur], h->cells[h->cur ^ 1], h->shift_table);
    h->cur ^= 1;
    h->shifts += 1;
    return cuda_code(cudaGetLastError());
}

int hdmc_sample(hdmc_t* h) {
    if (!h) return HDMC_EINVAL;
    const LaunchCtx c = h->ctx(h->stream);
    if (h->prec == HDMC_FP64) launch_hist_f64(c, h->cells[h->cur]);
    else launch_hist_f32(c, h->cells[h->cur]);
    h->n_samples += 1;
    return cuda_code(cudaGetLastError());
}

int hdmc_pressure(hdmc_t* h, double* betaP_over_rho, double* g_contact, uint64_t* hist, int64_t* n_samples) {
    if (!h) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // a strip's histogram: hdmc_strip_histogram
    int e = HDMC_OK;
    if (h->n_samples == 0) e = hdmc_sample(h);
    if (!e) e = check_device(h);
    if (e) return e;
    unsigned long long hh[kHistBins];
    e = cuda_code(cudaMemcpy(hh, h->hist, sizeof(hh), cudaMemcpyDeviceToHost));
    if (!e) e = cuda_code(cudaMemsetAsync(h->hist, 0, sizeof(hh), h->stream));
    if (e) return e;
    const int64_t ns = h->n_samples;
    h->n_samples = 0;
    double g0;
    const double bp = pressure_from_hist(h->desc(), hh, ns, &g0);
    if (betaP_over_rho) *betaP_over_rho = bp;
    if (g_contact) *g_contact = g0;
    if (hist)
        for (int i = 0; i < kHistBins; ++i) hist[i] = hh[i];
    if (n_samples) *n_samples = ns;
    return HDMC_OK;
}

int hdmc_psi6(hdmc_t* h, double r_cut, double out[4], double* psi) {
    if (!h || !out) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    const double wmin = h->prec == HDMC_FP64 ? std::min(h->g.wx, h->g.wy)
                                             : std::min((double)h->g.wxf, (double)h->g.wyf);
    if (!(r_cut > 0.0) || !(r_cut <= 2.0 * wmin)) return HDMC_EINVAL;
    const unsigned nb = psi6_blocks(h->g);
    // block sums go to the idle half of the double buffer (scratch between sweeps)
    if (sizeof(double) * 4 * (size_t)nb > h->lay.cells) return HDMC_EINVAL;
    double* partial = reinterpret_cast<double*>(h->cells[h->cur ^ 1]);
    const size_t psi_bytes = sizeof(double) * 8 * (size_t)h->g.C;
    double* dpsi = nullptr;
    int e = psi ? cuda_code(cudaMalloc((void**)&dpsi, psi_bytes)) : HDMC_OK;
    if (e) return e;
    const LaunchCtx c = h->ctx(h->stream);
    const double rc2 = r_cut * r_cut;
    if (h->prec == HDMC_FP64) launch_psi6_f64(c, h->cells[h->cur], rc2, dpsi, partial);
    else launch_psi6_f32(c, h->cells[h->cur], rc2, dpsi, partial);
    e = cuda_code(cudaGetLastError());
    std::vector<double> part(4 * (size_t)nb);
    if (!e)
        e = cuda_code(cudaMemcpyAsync(part.data(), partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                      h->stream));
    if (!e && psi) e = cuda_code(cudaMemcpyAsync(psi, dpsi, psi_bytes, cudaMemcpyDeviceToHost, h->stream));
    if (!e) e = cuda_code(cudaStreamSynchronize(h->stream));
    if (dpsi) cudaFree(dpsi);
    if (e) return e;
    double sum[4] = {0, 0, 0, 0};
    for (unsigned b = 0; b < nb; ++b)
        for (int k = 0; k < 4; ++k) sum[k] += part[4 * (size_t)b + k];
    for (int k = 0; k < 4; ++k) out[k] = sum[k] / (double)h->N;
    return check_device(h);
}

int hdmc_positions(hdmc_t* h, double* xy, int32_t* cell) {
    if (!h || !xy) return HDMC_EINVAL;
    if (h->nstrips) return HDMC_EINVAL;   // strips sweep in two phases (hdmc_strip_*)
    HostState hs;
    int e = download(h, hs);
    DevState ds;
    if (!e) e = read_devstate(h, ds);
    if (e) return e;
    const Geometry& g = h->g;
    const double wx = h->prec == HDMC_FP64 ? g.wx : (double)g.wxf;
    const double wy = h->prec == HDMC_FP64 ? g.wy : (double)g.wyf;
    const double Lx = h->prec == HDMC_FP64 ? h->Lx : (double)g.mx * wx;
    const double Ly = h->prec == HDMC_FP64 ? h->Ly : (double)g.my * wy;
    int64_t p = 0;
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            for (int j = 0; j < hs.cnt[c]; ++j) {
                if (p >= h->N) return HDMC_EOVERFLOW;
                double gx = ds.origin[0] + ((double)cx * wx + hs.loc[2 * (4 * c + j)]);
                double gy = ds.origin[1] + ((double)cy * wy + hs.loc[2 * (4 * c + j) + 1]);
                gx = gx - Lx * std::floor(gx / Lx);
                gy = gy - Ly * std::floor(gy / Ly);
                xy[2 * p] = gx;
                xy[2 * p + 1] = gy;
                if (cell) cell[p] = (int32_t)c;
                ++p;
            }
        }
    return p == h->N ? HDMC_OK : HDMC_EOVERFLOW;
}

int hdmc_get_state(hdmc_t* h, double* local, uint8_t* counts) {
    if (!h) return HDMC_EINVAL;
    HostState hs;
    int e = download(h, hs);
    if (e) return e;
    if (local) std::memcpy(local, hs.loc.data(), sizeof(double) * hs.loc.size());
    if (counts) std::memcpy(counts, hs.cnt.data(), hs.cnt.size());
    return check_device(h);
}

int hdmc_set_state(hdmc_t* h, const double* local, const uint8_t* counts, const double origin[2],
                   uint64_t sweeps_done, uint64_t shifts_done) {
    if (!h || !local || !counts || !origin) return HDMC_EINVAL;
    if (h && h->nstrips) return HDMC_EINVAL;
    HostState hs;
    int e = state_from_local(h->desc(), local, counts, hs);
    if (e) return e;
    e = cuda_code(cudaStreamSynchronize(h->stream));
    if (!e) e = upload(h, hs);
    DevState ds;
    if (!e) e = read_devstate(h, ds);
    if (e) return e;
    ds.origin[0] = origin[0];
    ds.origin[1] = origin[1];
    ds.sweep_next = sweeps_done;
    ds.shift_next = shifts_done;
    ds.error = 0;
    e = cuda_code(cudaMemcpy(h->st, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    if (!e) e = cuda_code(cudaDeviceSynchronize());   // as in hdmc_set_positions
    h->sweeps = sweeps_done;
    h->shifts = shifts_done;
    return e;
}

// ---- snapshots ------------------------------------------------------------------------
namespace {

constexpr char kSnapMagic[8] = {'H', 'D', 'M', 'C', 'S', 'N', 'P', '1'};
constexpr uint32_t kSnapVersion = 1;
constexpr size_t kSnapHeader = 256;

struct SnapHeader {
    char magic[8];
    uint32_t version, precision;
    int64_t N;
    double Lx, Ly, sigma, d;
    int32_t nsel, mx, my, nblocks;
    uint32_t key0, key1, flags, pad;
    uint64_t sweeps, shifts;
    int64_t n_samples;
    uint64_t off_state, off_partial, off_hist, off_cells, total;
};
static_assert(sizeof(SnapHeader) <= kSnapHeader, "snapshot header");

struct SnapLayout {
    size_t state, partial, hist, cells, cell_bytes, total;
};

SnapLayout snap_layout(const hdmc_t* h) {
    SnapLayout L;
    size_t p = kSnapHeader;
    L.state = p;
    p += align_up(sizeof(DevState));
    L.partial = p;
    p += align_up(sizeof(unsigned long long) * 4 * (size_t)h->lay.nblocks);
    L.hist = p;
    p += align_up(sizeof(unsigned long long) * kHistBins);
    L.cells = p;
    L.cell_bytes = (size_t)h->g.C * kSlots * (h->prec == HDMC_FP64 ? sizeof(double2) : sizeof(float2));
    L.total = p + L.cell_bytes;
    return L;
}

}  // namespace

size_t hdmc_snapshot_bytes(const hdmc_t* h) { return h ? snap_layout(h).total : 0; }

int hdmc_save(hdmc_t* h, void* buf, size_t bytes) {
    if (h && h->nstrips) return HDMC_EINVAL;
    if (!h || !buf) return HDMC_EINVAL;
    const SnapLayout L = snap_layout(h);
    if (bytes < L.total) return HDMC_EINVAL;
    char* b = static_cast<char*>(buf);
    SnapHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kSnapMagic, sizeof(kSnapMagic));
    hd.version = kSnapVersion;
    hd.precision = (uint32_t)h->prec;
    hd.N = h->N;
    hd.Lx = h->Lx;
    hd.Ly = h->Ly;
    hd.sigma = h->g.sigma;
    hd.d = h->g.d;
    hd.nsel = h->g.nsel;
    hd.mx = h->g.mx;
    hd.my = h->g.my;
    hd.nblocks = h->lay.nblocks;
    hd.key0 = h->g.key0;
    hd.key1 = h->g.key1;
    hd.flags = h->g.flags;
    hd.sweeps = h->sweeps;
    hd.shifts = h->shifts;
    hd.n_samples = h->n_samples;
    hd.off_state = L.state;
    hd.off_partial = L.partial;
    hd.off_hist = L.hist;
    hd.off_cells = L.cells;
    hd.total = L.total;
    std::memset(b, 0, L.cells);
    std::memcpy(b, &hd, sizeof(hd));
    const cudaStream_t s = h->stream;
    int e = cuda_code(cudaMemcpyAsync(b + L.state, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(b + L.partial, h->partial, sizeof(unsigned long long) * 4 * h->lay.nblocks,
                                      cudaMemcpyDeviceToHost, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(b + L.hist, h->hist, sizeof(unsigned long long) * kHistBins,
                                      cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaMemcpyAsync(b + L.cells, h->cells[h->cur], L.cell_bytes, cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    DevState ds;
    std::memcpy(&ds, b + L.state, sizeof(ds));
    return error_code(ds.error);
}

int hdmc_load(hdmc_t* h, const void* buf, size_t bytes) {
    if (h && h->nstrips) return HDMC_EINVAL;
    if (!h || !buf) return HDMC_EINVAL;
    const SnapLayout L = snap_layout(h);
    if (bytes < L.total) return HDMC_EINVAL;
    const char* b = static_cast<const char*>(buf);
    SnapHeader hd;
    std::memcpy(&hd, b, sizeof(hd));
    const Geometry& g = h->g;
    const bool same = std::memcmp(hd.magic, kSnapMagic, sizeof(kSnapMagic)) == 0 && hd.version == kSnapVersion &&
                      hd.precision == (uint32_t)h->prec && hd.N == h->N && hd.Lx == h->Lx && hd.Ly == h->Ly &&
                      hd.sigma == g.sigma && hd.mx == g.mx && hd.my == g.my && hd.nblocks == h->lay.nblocks &&
                      hd.off_state == L.state && hd.off_partial == L.partial && hd.off_hist == L.hist &&
                      hd.off_cells == L.cells && hd.total == L.total;
    if (!same) return HDMC_EINVAL;
    if (hd.nsel < 1 || hd.nsel > 255 || !(hd.d > 0) || !(hd.d < 0.5 * g.wx) || !(hd.d < 0.5 * g.wy) ||
        hd.n_samples < 0 || (hd.flags & ~(kNoParticleShuffle | kNoSetShuffle)) != 0)
        return HDMC_EINVAL;
    DevState ds;
    std::memcpy(&ds, b + L.state, sizeof(ds));
    if (ds.error != 0 || !std::isfinite(ds.origin[0]) || !std::isfinite(ds.origin[1])) return HDMC_EINVAL;

    // cells: into the idle half of the double buffer, checked there
    const cudaStream_t s = h->stream;
    const LaunchCtx c = h->ctx(s);
    void* idle = h->cells[h->cur ^ 1];
    unsigned long long res[2] = {0, 0};
    int e = cuda_code(cudaMemsetAsync(h->check, 0, 2 * sizeof(unsigned long long), s));
    if (!e) e = cuda_code(cudaMemcpyAsync(idle, b + L.cells, L.cell_bytes, cudaMemcpyHostToDevice, s));
    if (!e) {
        if (h->prec == HDMC_FP64) launch_check_f64(c, idle, h->check);
        else launch_check_f32(c, idle, h->check);
        e = cuda_code(cudaGetLastError());
    }
    if (!e) e = cuda_code(cudaMemcpyAsync(res, h->check, sizeof(res), cudaMemcpyDeviceToHost, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    if (res[1] != 0 || res[0] != (unsigned long long)h->N) return HDMC_EINVAL;

    // commit
    e = cuda_code(cudaMemcpyAsync(h->st, b + L.state, sizeof(DevState), cudaMemcpyHostToDevice, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(h->partial, b + L.partial, sizeof(unsigned long long) * 4 * h->lay.nblocks,
                                      cudaMemcpyHostToDevice, s));
    if (!e)
        e = cuda_code(cudaMemcpyAsync(h->hist, b + L.hist, sizeof(unsigned long long) * kHistBins,
                                      cudaMemcpyHostToDevice, s));
    if (!e) e = cuda_code(cudaStreamSynchronize(s));
    if (e) return e;
    h->cur ^= 1;
    h->sweeps = hd.sweeps;
    h->shifts = hd.shifts;
    h->n_samples = hd.n_samples;
    if (hd.d != g.d || hd.nsel != g.nsel || hd.key0 != g.key0 || hd.key1 != g.key1 || hd.flags != g.flags) {
        h->g.flags = hd.flags;
        h->g.d = hd.d;
        h->g.df = (float)hd.d;
        h->g.nsel = hd.nsel;
        h->g.key0 = hd.key0;
        h->g.key1 = hd.key1;
        h->drop_graphs();   // recorded kernels carry the old parameters
    }
    return HDMC_OK;
}

int hdmc_counters(hdmc_t* h, uint64_t out[4]) {
    if (!h || !out) return HDMC_EINVAL;
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    if (e) return e;
    std::vector<unsigned long long> part(4 * (size_t)h->lay.nblocks);
    e = cuda_code(cudaMemcpy(part.data(), h->partial, sizeof(unsigned long long) * part.size(),
                             cudaMemcpyDeviceToHost));
    if (e) return e;
    for (int k = 0; k < 4; ++k) out[k] = 0;
    for (size_t b = 0; b < (size_t)h->lay.nblocks; ++b)
        for (int k = 0; k < 4; ++k) out[k] += part[4 * b + k];
    return check_device(h);
}

int hdmc_info(hdmc_t* h, int32_t* mx, int32_t* my, double* wx, double* wy, uint64_t* sweeps_done,
              uint64_t* shifts_done, double origin[2]) {
    if (!h) return HDMC_EINVAL;
    if (mx) *mx = h->g.mx;
    if (my) *my = h->g.my;
    if (wx) *wx = h->g.wx;
    if (wy) *wy = h->g.wy;
    if (sweeps_done) *sweeps_done = h->sweeps;
    if (shifts_done) *shifts_done = h->shifts;
    if (origin) {
        DevState ds;
        const int e = read_devstate(h, ds);
        if (e) return e;
        origin[0] = ds.origin[0];
        origin[1] = ds.origin[1];
    }
    return HDMC_OK;
}

int hdmc_set_move_size(hdmc_t* h, double d) {
    if (!h || !(d > 0) || !(d < 0.5 * h->g.wx) || !(d < 0.5 * h->g.wy)) return HDMC_EINVAL;
    h->g.d = d;
    h->g.df = (float)d;
    h->drop_graphs();   // recorded kernels carry the old value
    return HDMC_OK;
}

int hdmc_set_balance(hdmc_t* h, int shuffle_particles, int shuffle_sets) {
    if (!h) return HDMC_EINVAL;
    const uint32_t f = (shuffle_particles ? 0u : kNoParticleShuffle) | (shuffle_sets ? 0u : kNoSetShuffle);
    if (f != h->g.flags) {
        h->g.flags = f;
        h->drop_graphs();   // recorded kernels carry the old geometry
    }
    return HDMC_OK;
}

int hdmc_tune_move_size(hdmc_t* h, double target, int64_t sweeps, int64_t every, double* d_out) {
    if (!h || !(target > 0.0) || !(target < 1.0) || sweeps < 1 || every < 1) return HDMC_EINVAL;
    const double dmax = 0.49 * std::min(h->g.wx, h->g.wy);
    const double dmin = 1e-6 * h->g.sigma;
    uint64_t c0[4], c1[4];
    int e = hdmc_counters(h, c0);
    for (int64_t done = 0; !e && done < sweeps; done += every) {
        e = hdmc_sweep(h, std::min(every, sweeps - done));
        if (!e) e = hdmc_counters(h, c1);
        if (e) break;
        const uint64_t tr = c1[0] - c0[0], ac = c1[1] - c0[1];
        double f = 2.0;
        if (tr > 0) f = std::sqrt(((double)ac / (double)tr) / target);
        f = std::min(std::max(f, 0.5), 2.0);
        const double d = std::min(std::max(h->g.d * f, dmin), dmax);
        e = hdmc_set_move_size(h, d);
        for (int k = 0; k < 4; ++k) c0[k] = c1[k];
    }
    if (!e && d_out) *d_out = h->g.d;
    return e;
}

int hdmc_set_stream(hdmc_t* h, void* stream) {
    if (!h) return HDMC_EINVAL;
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)stream;
    return e;
}

int hdmc_sync(hdmc_t* h) {
    if (!h) return HDMC_EINVAL;
    return check_device(h);
}

void hdmc_destroy(hdmc_t* h) {
    if (!h) return;
    if (h->stream || h->ws) cudaStreamSynchronize(h->stream);
    h->drop_graphs();
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    delete h;
}

// ---- spatial decomposition with inactive bands (Sec. 6) ---------------------------
namespace {

// First row of strip k of R: 2 floor(k my / (2R)) (even, so every strip
// starts on the same checkerboard parity; every strip has >= 2 rows).
int strip_start(int my, int R, int k) { return 2 * (int)(((int64_t)k * my) / (2 * (int64_t)R)); }

// Local row of a strip handle holding global row gy: rows r0-2 .. r1+1 are
// local rows 0 .. my-1 (periodic in the global rows).
int strip_local_row(const hdmc_t* h, int which) {
    const int own = h->r1 - h->r0;
    switch (which) {   // own edge rows r0, r0+1, r1-2, r1-1 / halo rows r0-2, r0-1, r1, r1+1
        case 0: return 2;
        case 1: return 3;
        case 2: return own;
        case 3: return own + 1;
        case 4: return 0;
        case 5: return 1;
        case 6: return own + 2;
        case 7: return own + 3;
        default: return -1;
    }
}

// Copies local row ly between the current cell buffer and buf (host or
// device memory): the row's even-x cells then its odd-x cells, each a
// contiguous run of mx/2 cells of the set-major layout.
int strip_copy_row(hdmc_t* h, int ly, void* buf, bool to_buf) {
    const Geometry& g = h->g;
    const size_t el = h->prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    const size_t half = (size_t)g.hx * 8 * el;
    char* cells = (char*)h->cells[h->cur];
    int e = HDMC_OK;
    for (int p = 0; p < 2 && !e; ++p) {
        const long long s0 = storage_index(g, p, ly);   // first cell of the half row
        char* dev = cells + (size_t)s0 * 8 * el;
        char* b = (char*)buf + p * half;
        e = cuda_code(to_buf ? cudaMemcpyAsync(b, dev, half, cudaMemcpyDefault, h->stream)
                             : cudaMemcpyAsync(dev, b, half, cudaMemcpyDefault, h->stream));
    }
    if (!e) e = cuda_code(cudaStreamSynchronize(h->stream));
    return e;
}

}  // namespace

int hdmc_strip_create(hdmc_t** out, int64_t N, double Lx, double Ly, double sigma, double d, int nselect,
                      uint64_t seed, int precision, int32_t nstrips, int32_t strip, void* stream) {
    if (!out) return HDMC_EINVAL;
    *out = nullptr;
    if (N < 2 || (N & 1)) return HDMC_EINVAL;
    SysDesc G;
    int e = make_system(G, N, Lx, Ly, sigma, d, nselect, seed, precision);
    if (e) return e;
    if (nstrips < 1 || strip < 0 || strip >= nstrips || G.g.my < 2 * nstrips) return HDMC_EINVAL;
    HostState whole;
    e = start_state(G, whole);
    if (e) return e;
    hdmc_t* h = new (std::nothrow) hdmc_t();
    if (!h) return HDMC_ENOMEM;
    h->nstrips = nstrips;
    h->strip = strip;
    h->myg = G.g.my;
    h->r0 = strip_start(G.g.my, nstrips, strip);
    h->r1 = strip + 1 == nstrips ? G.g.my : strip_start(G.g.my, nstrips, strip + 1);
    const int own = h->r1 - h->r0;
    Geometry g = G.g;
    g.my = own + 4;   // two halo rows on either side; even, as own is
    g.hy = g.my / 2;
    g.cq = (long long)g.hx * g.hy;
    g.C = (long long)g.mx * g.my;
    g.row0 = h->r0 - 2;
    g.ylo = 3;          // the strip's first row (global r0) is its inactive band
    g.yhi = own + 1;
    g.slo = 2;
    g.shi = own + 1;
    h->g = g;
    h->Lx = Lx;
    h->Ly = Ly;
    h->prec = G.prec;
    h->stream = (cudaStream_t)stream;
    h->lay = make_layout(g, G.prec);
    // the strip's rows and halos of the whole start configuration
    HostState hs;
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign((size_t)g.C, 0);
    int64_t mine = 0;
    for (int ly = 0; ly < g.my; ++ly) {
        const int gy = ((g.row0 + ly) % G.g.my + G.g.my) % G.g.my;
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)ly * g.mx + cx, gc = (int64_t)gy * g.mx + cx;
            hs.cnt[c] = whole.cnt[gc];
            for (int k = 0; k < 8; ++k) hs.loc[8 * c + k] = whole.loc[8 * gc + k];
            if (ly >= 2 && ly <= own + 1) mine += whole.cnt[gc];
        }
    }
    h->N = mine;
    e = cuda_code(cudaMalloc((void**)&h->ws, h->lay.total));
    h->own_ws = e == HDMC_OK;
    if (!e) e = cuda_code(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    if (e) {
        hdmc_destroy(h);
        return e;
    }
    char* p = h->ws;
    h->cells[0] = p;
    p += h->lay.cells;
    h->cells[1] = p;
    p += h->lay.cells;
    h->table = (SweepDraw*)p;
    p += h->lay.table;
    h->shift_table = (SweepDraw*)p;
    p += h->lay.shift_table;
    h->st = (DevState*)p;
    h->g.check = &h->st->error;
    p += h->lay.state;
    h->partial = (unsigned long long*)p;
    p += h->lay.partial;
    h->hist = (unsigned long long*)p;
    p += h->lay.hist;
    h->edges2 = (double*)p;
    p += h->lay.edges;
    h->check = (unsigned long long*)p;
    e = cuda_code(cudaMemset(h->ws + 2 * h->lay.cells, 0, h->lay.total - 2 * h->lay.cells));
    if (!e) {
        double E[kHistBins + 1];
        squared_edges(sigma, E);
        e = cuda_code(cudaMemcpy(h->edges2, E, sizeof(E), cudaMemcpyHostToDevice));
    }
    if (!e) e = upload(h, hs);
    if (!e) e = cuda_code(cudaDeviceSynchronize());
    if (e) {
        hdmc_destroy(h);
        return e;
    }
    *out = h;
    return HDMC_OK;
}

int hdmc_strip_rows(hdmc_t* h, int32_t* first_row, int32_t* end_row) {
    if (!h || !h->nstrips) return HDMC_EINVAL;
    if (first_row) *first_row = h->r0;
    if (end_row) *end_row = h->r1;
    return HDMC_OK;
}

int hdmc_strip_subsweeps(hdmc_t* h) {
    if (!h || !h->nstrips || h->pending) return HDMC_EINVAL;
    LaunchCtx c = h->ctx(h->stream);
    launch_draws(c, h->table, 1, true);
    for (int k = 0; k < 4; ++k) {
        if (h->prec == HDMC_FP64) launch_subsweep_f64(c, h->cells[h->cur], h->table, k);
        else launch_subsweep_f32(c, h->cells[h->cur], h->table, k);
    }
    h->pending = true;
    return cuda_code(cudaGetLastError());
}

int hdmc_strip_shift(hdmc_t* h) {
    if (!h || !h->nstrips || !h->pending) return HDMC_EINVAL;
    const LaunchCtx c = h->ctx(h->stream);
    if (h->prec == HDMC_FP64) launch_shift_f64(c, h->cells[h->cur], h->cells[h->cur ^ 1], h->table);
    else launch_shift_f32(c, h->cells[h->cur], h->cells[h->cur ^ 1], h->table);
    h->cur ^= 1;
    h->sweeps += 1;
    h->pending = false;
    return cuda_code(cudaGetLastError());
}

size_t hdmc_strip_row_bytes(const hdmc_t* h) {
    if (!h || !h->nstrips) return 0;
    return (size_t)h->g.mx * 8 * (h->prec == HDMC_FP64 ? sizeof(double) : sizeof(float));
}

int hdmc_strip_get_row(hdmc_t* h, int32_t which, void* buf) {
    if (!h || !h->nstrips || !buf || which < 0 || which > 3) return HDMC_EINVAL;
    return strip_copy_row(h, strip_local_row(h, which), buf, true);
}

int hdmc_strip_set_halo(hdmc_t* h, int32_t which, const void* buf) {
    if (!h || !h->nstrips || !buf || which < 0 || which > 3) return HDMC_EINVAL;
    return strip_copy_row(h, strip_local_row(h, which + 4), const_cast<void*>(buf), false);
}

int hdmc_strip_histogram(hdmc_t* h, uint64_t* hist, int64_t* n_samples) {
    if (!h || !h->nstrips || !hist) return HDMC_EINVAL;
    int e = check_device(h);
    if (e) return e;
    unsigned long long hh[kHistBins];
    e = cuda_code(cudaMemcpy(hh, h->hist, sizeof(hh), cudaMemcpyDeviceToHost));
    if (!e) e = cuda_code(cudaMemsetAsync(h->hist, 0, sizeof(hh), h->stream));
    if (!e) e = cuda_code(cudaStreamSynchronize(h->stream));
    if (e) return e;
    for (int i = 0; i < kHistBins; ++i) hist[i] = hh[i];
    if (n_samples) *n_samples = h->n_samples;
    h->n_samples = 0;
    return HDMC_OK;
}

int hdmc_pressure_fit(const uint64_t* hist, int64_t n_samples, int64_t N, double Lx, double Ly, double sigma,
                      double* betaP_over_rho, double* g_contact) {
    if (!hist || n_samples < 1 || N < 1 || !(Lx > 0) || !(Ly > 0) || !(sigma > 0)) return HDMC_EINVAL;
    SysDesc d{};
    d.g.sigma = sigma;
    d.g.sig2 = sigma * sigma;
    d.N = N;
    d.Lx = Lx;
    d.Ly = Ly;
    unsigned long long hh[kHistBins];
    for (int i = 0; i < kHistBins; ++i) hh[i] = hist[i];
    double g0;
    const double bp = pressure_from_hist(d, hh, n_samples, &g0);
    if (betaP_over_rho) *betaP_over_rho = bp;
    if (g_contact) *g_contact = g0;
    return HDMC_OK;
}

int hdmc_build_flags(void) {
#ifdef HDMC_CHECK
    return HDMC_BUILD_CHECK;
#else
    return 0;
#endif
}

const char* hdmc_strerror(int code) {
    switch (code) {
        case HDMC_OK: return "ok";
        case HDMC_EINVAL: return "invalid argument";
        case HDMC_ECUDA: return "CUDA runtime error";
        case HDMC_EOVERFLOW: return "more disks or spheres in a cell than it has slots";
        case HDMC_EOVERLAP: return "overlapping disks";
        case HDMC_ETIMEOUT: return "bounded device wait timed out";
        case HDMC_ENOMEM: return "out of memory or workspace too small";
        case HDMC_ECHECK: return "a kernel computed a cell index outside the grid (checked build)";
        default: return "unknown error";
    }
}

}  // extern "C"
