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

using namespace hdmc;

namespace {

constexpr int kChunk = 64;       // sweeps per recorded graph
constexpr size_t kAlign = 256;   // workspace segment alignment

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Cell grid of a box: mx = largest even integer <= Lx/sigma (likewise my),
// w = L/m; needs m >= 4 and w < sqrt(2) sigma (at most 4 disks per cell).
bool make_grid(double Lx, double Ly, double sigma, int& mx, int& my, double& wx, double& wy) {
    if (!(sigma > 0) || !(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly)) return false;
    const double qx = std::floor(Lx / sigma), qy = std::floor(Ly / sigma);
    if (qx > 1.0e9 || qy > 1.0e9) return false;
    mx = (int)qx;
    my = (int)qy;
    mx -= mx & 1;
    my -= my & 1;
    if (mx < 4 || my < 4) return false;
    wx = Lx / mx;
    wy = Ly / my;
    return wx * wx < 2.0 * sigma * sigma && wy * wy < 2.0 * sigma * sigma;
}

struct Layout {
    size_t cells, table, shift_table, state, partial, hist, edges, total;
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
    L.total = 2 * L.cells + L.table + L.shift_table + L.state + L.partial + L.hist + L.edges;
    return L;
}

int cuda_code(cudaError_t e) {
    if (e == cudaSuccess) return HDMC_OK;
    if (e == cudaErrorMemoryAllocation) return HDMC_ENOMEM;
    return HDMC_ECUDA;
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
    uint64_t sweeps = 0, shifts = 0;
    int64_t n_samples = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (sweeps, parity) -> graph

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
};

namespace {

// ---- start configuration and binning -----------------------------------------

// Hexagonal patch nx x ny (ny even, nx*ny = N) whose row spacing is closest,
// in ratio, to sqrt(3)/2 of its column spacing.
bool lattice_shape(int64_t N, double Lx, double Ly, int64_t& nx, int64_t& ny) {
    nx = ny = -1;
    double best = 0;
    for (int64_t r = 2; r <= N; r += 2) {
        if (N % r) continue;
        const int64_t c = N / r;
        const double cost = std::fabs(std::log((Ly / (double)r) / ((Lx / (double)c) * 0.86602540378443864676)));
        if (nx < 0 || cost < best) {
            best = cost;
            nx = c;
            ny = r;
        }
    }
    return nx > 0;
}

// Site p = j*nx + i at ((i + 1/2 + (j mod 2)/2) Lx/nx, (j + 1/2) Ly/ny), moved by
// a uniform point of the disk of radius 0.01 sigma (start stream of p).
void lattice_positions(int64_t N, double Lx, double Ly, double sigma, uint32_t k0, uint32_t k1, int64_t nx,
                       int64_t ny, std::vector<double>& xy) {
    xy.resize(2 * (size_t)N);
    const double ax = Lx / (double)nx, ay = Ly / (double)ny, rj = 0.01 * sigma;
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            const int64_t p = j * nx + i;
            const double x0 = ((double)i + 0.5 + 0.5 * (double)(j & 1)) * ax;
            const double y0 = ((double)j + 0.5) * ay;
            WordStream s(k0, k1, (uint32_t)p, 0xFFFFFFFEu, kDomInit << 28);
            double u, v;
            for (;;) {
                const uint32_t a = s.next(), b = s.next(), c = s.next(), e = s.next();
                u = sym52(a, b);
                v = sym52(c, e);
                if (u * u + v * v < 1.0) break;
            }
            double x = x0 + rj * u, y = y0 + rj * v;
            if (x >= Lx) x -= Lx;
            if (x < 0.0) x += Lx;
            if (y >= Ly) y -= Ly;
            if (y < 0.0) y += Ly;
            xy[2 * p] = x;
            xy[2 * p + 1] = y;
        }
}

// Cell of a coordinate: trunc(x/w) clamped, corrected by one cell when the
// rounded local offset falls outside [0,w), then the offset clamped into it.
void bin_axis(double x, double w, int m, int& cell, double& loc) {
    int c = (int)(x / w);
    c = std::min(std::max(c, 0), m - 1);
    double l = x - (double)c * w;
    if (l < 0.0 && c > 0) {
        c -= 1;
        l = x - (double)c * w;
    }
    if (l >= w && c < m - 1) {
        c += 1;
        l = x - (double)c * w;
    }
    if (l < 0.0) l = 0.0;
    if (l >= w) l = std::nextafter(w, 0.0);
    cell = c;
    loc = l;
}

// Canonical host copy of a state: loc[(4c+j)*2+k], cnt[c].
struct HostState {
    std::vector<double> loc;
    std::vector<uint8_t> cnt;
};

int bin_positions(const hdmc_t* h, const double* xy, HostState& hs) {
    const Geometry& g = h->g;
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign((size_t)g.C, 0);
    for (int64_t p = 0; p < h->N; ++p) {
        const double x = xy[2 * p], y = xy[2 * p + 1];
        if (!(x >= 0.0 && x <= h->Lx && y >= 0.0 && y <= h->Ly)) return HDMC_EINVAL;
        int cx, cy;
        double lx, ly;
        bin_axis(x, g.wx, g.mx, cx, lx);
        bin_axis(y, g.wy, g.my, cy, ly);
        const int64_t c = (int64_t)cy * g.mx + cx;
        if (hs.cnt[c] >= kSlots) return HDMC_EOVERFLOW;
        const int j = hs.cnt[c]++;
        if (h->prec == HDMC_FP32_LOCAL) {
            float fx = (float)lx, fy = (float)ly;
            if (fx >= g.wxf) fx = std::nextafter(g.wxf, 0.0f);
            if (fy >= g.wyf) fy = std::nextafter(g.wyf, 0.0f);
            lx = fx;
            ly = fy;
        }
        hs.loc[2 * (4 * c + j)] = lx;
        hs.loc[2 * (4 * c + j) + 1] = ly;
    }
    return HDMC_OK;
}

// Overlap test of every disk against its 3x3 neighbourhood, in cell-local
// frames with the arithmetic of the sweep.
bool any_overlap(const hdmc_t* h, const HostState& hs) {
    const Geometry& g = h->g;
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            for (int i = 0; i < hs.cnt[c]; ++i) {
                const double px = hs.loc[2 * (4 * c + i)], py = hs.loc[2 * (4 * c + i) + 1];
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int ncx = (cx + dx + g.mx) % g.mx, ncy = (cy + dy + g.my) % g.my;
                        const int64_t nc = (int64_t)ncy * g.mx + ncx;
                        for (int j = 0; j < hs.cnt[nc]; ++j) {
                            if (dx == 0 && dy == 0 && i == j) continue;
                            const double qx = hs.loc[2 * (4 * nc + j)], qy = hs.loc[2 * (4 * nc + j) + 1];
                            if (h->prec == HDMC_FP64) {
                                const double ex = qx + (double)dx * g.wx, ey = qy + (double)dy * g.wy;
                                const double ddx = px - ex, ddy = py - ey;
                                if (ddx * ddx + ddy * ddy < g.sig2) return true;
                            } else {
                                const float ex = (float)qx + (float)dx * g.wxf, ey = (float)qy + (float)dy * g.wyf;
                                const float ddx = (float)px - ex, ddy = (float)py - ey;
                                if (std::fma(ddx, ddx, std::fma(ddy, ddy, -g.sig2f)) < 0.0f) return true;
                            }
                        }
                    }
            }
        }
    return false;
}

// Canonical host state <-> set-major device cells (x0..x3 then y0..y3 per cell).
void pack(const hdmc_t* h, const HostState& hs, std::vector<char>& raw) {
    const Geometry& g = h->g;
    const size_t el = h->prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    raw.assign((size_t)g.C * 8 * el, 0);
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            const long long s = storage_index(g, cx, cy);
            for (int j = 0; j < kSlots; ++j) {
                const double x = j < hs.cnt[c] ? hs.loc[2 * (4 * c + j)] : kEmpty;
                const double y = j < hs.cnt[c] ? hs.loc[2 * (4 * c + j) + 1] : kEmpty;
                if (h->prec == HDMC_FP64) {
                    std::memcpy(raw.data() + (8 * s + j) * el, &x, el);
                    std::memcpy(raw.data() + (8 * s + 4 + j) * el, &y, el);
                } else {
                    const float fx = (float)x, fy = (float)y;
                    std::memcpy(raw.data() + (8 * s + j) * el, &fx, el);
                    std::memcpy(raw.data() + (8 * s + 4 + j) * el, &fy, el);
                }
            }
        }
}

void unpack(const hdmc_t* h, const std::vector<char>& raw, HostState& hs) {
    const Geometry& g = h->g;
    const size_t el = h->prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign((size_t)g.C, 0);
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            const long long s = storage_index(g, cx, cy);
            int n = 0;
            for (int j = 0; j < kSlots; ++j) {
                double x, y;
                if (h->prec == HDMC_FP64) {
                    std::memcpy(&x, raw.data() + (8 * s + j) * el, el);
                    std::memcpy(&y, raw.data() + (8 * s + 4 + j) * el, el);
                } else {
                    float fx, fy;
                    std::memcpy(&fx, raw.data() + (8 * s + j) * el, el);
                    std::memcpy(&fy, raw.data() + (8 * s + 4 + j) * el, el);
                    x = fx;
                    y = fy;
                }
                if (x >= 0.0) n = j + 1;
                hs.loc[2 * (4 * c + j)] = x >= 0.0 ? x : kEmpty;
                hs.loc[2 * (4 * c + j) + 1] = x >= 0.0 ? y : kEmpty;
            }
            hs.cnt[c] = (uint8_t)n;
        }
}

int upload(hdmc_t* h, const HostState& hs) {
    std::vector<char> raw;
    pack(h, hs, raw);
    return cuda_code(cudaMemcpy(h->cells[h->cur], raw.data(), raw.size(), cudaMemcpyHostToDevice));
}

int download(hdmc_t* h, HostState& hs) {
    int e = cuda_code(cudaStreamSynchronize(h->stream));
    if (e) return e;
    std::vector<char> raw(h->lay.cells);
    e = cuda_code(cudaMemcpy(raw.data(), h->cells[h->cur], raw.size(), cudaMemcpyDeviceToHost));
    if (e) return e;
    unpack(h, raw, hs);
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
    return (ds.error & 1u) ? HDMC_EOVERFLOW : HDMC_OK;
}

// ---- sweep driver ------------------------------------------------------------

void enqueue_sweeps(hdmc_t* h, cudaStream_t s, int K, int parity) {
    const LaunchCtx c = h->ctx(s);
    launch_draws(c, h->table, K, true);
    for (int j = 0; j < K; ++j) {
        void* a = h->cells[parity ^ (j & 1)];
        void* b = h->cells[parity ^ (j & 1) ^ 1];
        for (int k = 0; k < 4; ++k) {
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

// ---- Sec. 4 pressure fit -------------------------------------------------------

// Least-squares polynomial of degree `deg` through (t_i, y_i) by Householder
// QR; returns the constant coefficient (the value at t = 0).
double poly_intercept(const std::vector<double>& t, const std::vector<double>& y, int deg) {
    const int n = (int)t.size(), p = deg + 1;
    std::vector<double> A((size_t)n * p), b(y);
    for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int k = 0; k < p; ++k) {
            A[(size_t)i * p + k] = v;
            v *= t[i];
        }
    }
    for (int k = 0; k < p; ++k) {
        double norm = 0.0;
        for (int i = k; i < n; ++i) norm += A[(size_t)i * p + k] * A[(size_t)i * p + k];
        norm = std::sqrt(norm);
        const double alpha = A[(size_t)k * p + k] > 0 ? -norm : norm;
        std::vector<double> v(n - k);
        for (int i = k; i < n; ++i) v[i - k] = A[(size_t)i * p + k];
        v[0] -= alpha;
        double vn = 0.0;
        for (double q : v) vn += q * q;
        if (vn == 0.0) continue;
        for (int c = k; c < p; ++c) {
            double s = 0.0;
            for (int i = k; i < n; ++i) s += v[i - k] * A[(size_t)i * p + c];
            s = 2.0 * s / vn;
            for (int i = k; i < n; ++i) A[(size_t)i * p + c] -= s * v[i - k];
        }
        double s = 0.0;
        for (int i = k; i < n; ++i) s += v[i - k] * b[i];
        s = 2.0 * s / vn;
        for (int i = k; i < n; ++i) b[i] -= s * v[i - k];
    }
    std::vector<double> a(p);
    for (int k = p - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < p; ++c) s -= A[(size_t)k * p + c] * a[c];
        a[k] = s / A[(size_t)k * p + k];
    }
    return a[0];
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================
extern "C" {

size_t hdmc_workspace_bytes(int64_t N, double Lx, double Ly, double sigma, int precision) {
    int mx, my;
    double wx, wy;
    if (N < 1 || (precision != HDMC_FP64 && precision != HDMC_FP32_LOCAL)) return 0;
    if (!make_grid(Lx, Ly, sigma, mx, my, wx, wy)) return 0;
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
    int mx, my;
    double wx, wy;
    if (N < 2 || (N & 1) || nselect < 1 || nselect > 255) return HDMC_EINVAL;
    if (precision != HDMC_FP64 && precision != HDMC_FP32_LOCAL) return HDMC_EINVAL;
    if (!make_grid(Lx, Ly, sigma, mx, my, wx, wy)) return HDMC_EINVAL;
    if (!(d > 0) || !(d < 0.5 * wx) || !(d < 0.5 * wy)) return HDMC_EINVAL;
    if ((int64_t)mx * my * kSlots < N) return HDMC_EINVAL;
    if (dev_workspace && ((uintptr_t)dev_workspace % kAlign)) return HDMC_EINVAL;

    hdmc_t* h = new (std::nothrow) hdmc_t();
    if (!h) return HDMC_ENOMEM;
    Geometry& g = h->g;
    g.mx = mx;
    g.my = my;
    g.hx = mx / 2;
    g.hy = my / 2;
    g.cq = (long long)g.hx * g.hy;
    g.C = (long long)mx * my;
    g.wx = wx;
    g.wy = wy;
    g.wxf = (float)wx;
    g.wyf = (float)wy;
    g.sigma = sigma;
    g.sig2 = sigma * sigma;
    g.sig2f = (float)(sigma * sigma);
    g.d = d;
    g.df = (float)d;
    g.nsel = nselect;
    g.key0 = (uint32_t)seed;
    g.key1 = (uint32_t)(seed >> 32);
    h->N = N;
    h->Lx = Lx;
    h->Ly = Ly;
    h->prec = precision;
    h->stream = (cudaStream_t)stream;
    h->lay = make_layout(g, precision);

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
    p += h->lay.state;
    h->partial = (unsigned long long*)p;
    p += h->lay.partial;
    h->hist = (unsigned long long*)p;
    p += h->lay.hist;
    h->edges2 = (double*)p;

    e = cuda_code(cudaMemset(h->ws + 2 * h->lay.cells, 0, h->lay.total - 2 * h->lay.cells));
    if (!e) {
        // squared histogram bin edges (sigma + k dr)^2, each rounded once
        double E[kHistBins + 1];
        const double dr = kHistDr * sigma;
        for (int k = 0; k <= kHistBins; ++k) {
            const double edge = sigma + (double)k * dr;
            E[k] = edge * edge;
        }
        e = cuda_code(cudaMemcpy(h->edges2, E, sizeof(E), cudaMemcpyHostToDevice));
    }
    int64_t nx, ny;
    if (!e && !lattice_shape(N, Lx, Ly, nx, ny)) e = HDMC_EINVAL;
    if (!e) {
        std::vector<double> xy;
        lattice_positions(N, Lx, Ly, sigma, g.key0, g.key1, nx, ny, xy);
        HostState hs;
        e = bin_positions(h, xy.data(), hs);
        if (!e && any_overlap(h, hs)) e = HDMC_EOVERLAP;
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
    HostState hs;
    int e = bin_positions(h, xy, hs);
    if (e) return e;
    if (any_overlap(h, hs)) return HDMC_EOVERLAP;
    e = cuda_code(cudaStreamSynchronize(h->stream));
    if (!e) e = upload(h, hs);
    DevState ds;
    if (!e) e = read_devstate(h, ds);
    if (!e) {
        ds.origin[0] = ds.origin[1] = 0.0;
        e = cuda_code(cudaMemcpy(h->st, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    }
    return e;
}

int hdmc_sweep(hdmc_t* h, int64_t n) {
    if (!h || n < 0) return HDMC_EINVAL;
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
    const int nev = 2;
    cudaEvent_t ev[nev];
    for (int i = 0; i < nev; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) return HDMC_ECUDA;
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

int hdmc_shift(hdmc_t* h) {
    if (!h) return HDMC_EINVAL;
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
    const double sigma = h->g.sigma, dr = kHistDr * sigma, c = kFitRange * sigma;
    const double rho = (double)h->N / (h->Lx * h->Ly);
    std::vector<double> t, gv;
    for (int i = 0; i < kHistBins; ++i) {
        const double r0 = sigma + dr * i, r1 = sigma + dr * (i + 1);
        const double R = (2.0 / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0) / (r1 * r1 - r0 * r0);   // Eq. R
        if (!(R > sigma && R <= sigma + c)) continue;
        const double gR = (double)hh[i] / ((double)ns * (double)h->N * rho * 2.0 * M_PI * R * dr);   // Eq. gR
        t.push_back((R - sigma) / c);
        gv.push_back(gR);
    }
    const double g0 = poly_intercept(t, gv, kFitDegree);
    if (betaP_over_rho) *betaP_over_rho = 1.0 + 0.5 * M_PI * rho * sigma * sigma * g0;   // Eq. P
    if (g_contact) *g_contact = g0;
    if (hist)
        for (int i = 0; i < kHistBins; ++i) hist[i] = hh[i];
    if (n_samples) *n_samples = ns;
    return HDMC_OK;
}

int hdmc_positions(hdmc_t* h, double* xy, int32_t* cell) {
    if (!h || !xy) return HDMC_EINVAL;
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
    const Geometry& g = h->g;
    HostState hs;
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign(counts, counts + g.C);
    int64_t total = 0;
    for (int64_t c = 0; c < g.C; ++c) {
        if (hs.cnt[c] > kSlots) return HDMC_EINVAL;
        total += hs.cnt[c];
        for (int j = 0; j < hs.cnt[c]; ++j) {
            const double x = local[2 * (4 * c + j)], y = local[2 * (4 * c + j) + 1];
            const bool fits = h->prec == HDMC_FP64 ? (x >= 0 && x < g.wx && y >= 0 && y < g.wy)
                                                   : ((double)(float)x == x && (double)(float)y == y && x >= 0 &&
                                                      (float)x < g.wxf && y >= 0 && (float)y < g.wyf);
            if (!fits) return HDMC_EINVAL;
            hs.loc[2 * (4 * c + j)] = x;
            hs.loc[2 * (4 * c + j) + 1] = y;
        }
    }
    if (total != h->N) return HDMC_EINVAL;
    int e = cuda_code(cudaStreamSynchronize(h->stream));
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
    h->sweeps = sweeps_done;
    h->shifts = shifts_done;
    return e;
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

const char* hdmc_strerror(int code) {
    switch (code) {
        case HDMC_OK: return "ok";
        case HDMC_EINVAL: return "invalid argument";
        case HDMC_ECUDA: return "CUDA runtime error";
        case HDMC_EOVERFLOW: return "more than 4 disks in a cell";
        case HDMC_EOVERLAP: return "overlapping disks";
        case HDMC_ETIMEOUT: return "bounded device wait timed out";
        case HDMC_ENOMEM: return "out of memory or workspace too small";
        default: return "unknown error";
    }
}

}  // extern "C"
