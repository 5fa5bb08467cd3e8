// hdmc_host.cu -- host-side helpers shared by the single-system and batch
// entry points: cell grid, hexagonal start, binning and the legality check of
// a configuration, conversion between the canonical state and the device
// cell layout, and the Sec. 4 pressure fit.  Compiled with
// -ffp-contract=off so the start configuration is the same on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hdmc_host.h"

namespace hdmc {

int cuda_code(cudaError_t e) {
    if (e == cudaSuccess) return HDMC_OK;
    if (e == cudaErrorMemoryAllocation) return HDMC_ENOMEM;
    return HDMC_ECUDA;
}

int error_code(unsigned int device_error) {
    if (device_error & kErrIndex) return HDMC_ECHECK;
    if (device_error & kErrOverflow) return HDMC_EOVERFLOW;
    return HDMC_OK;
}

// Cells along one axis of length L.  Default rule: m = largest even integer
// <= L/sigma (cells just wider than sigma).  HDMC_CELLS_SQRT2 (Sec. 3.1):
// floor(L/(sqrt(2) sigma)) rounded up to the smallest even m > L/(sqrt(2)
// sigma), the widest cells that still hold at most 4 centres (Fig. 3); it
// must not make w < sigma.  m is even so that the checkerboard tiles the
// periodic box (Eq. 1).  -1 if invalid.
static int cells_along(double L, double sigma, int rule) {
    const double q = std::floor(L / sigma);
    if (q > 1.0e9) return -1;
    int m = (int)q;
    m -= m & 1;
    if (rule == 1) {
        int k = (int)(std::floor(L / (std::sqrt(2.0) * sigma)) + 1.0);
        k += k & 1;
        if (k > m) return -1;
        m = k;
    }
    return m;
}

// Cell grid of a box: mx, my by the rule, w = L/m; needs m >= 4 and
// w < sqrt(2) sigma (at most 4 disks per cell).
bool make_grid(double Lx, double Ly, double sigma, int& mx, int& my, double& wx, double& wy, int rule) {
    if (!(sigma > 0) || !(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly)) return false;
    if (rule < 0 || rule > 1) return false;
    mx = cells_along(Lx, sigma, rule);
    my = cells_along(Ly, sigma, rule);
    if (mx < 4 || my < 4) return false;
    wx = Lx / mx;
    wy = Ly / my;
    return wx * wx < 2.0 * sigma * sigma && wy * wy < 2.0 * sigma * sigma;
}

int make_system(SysDesc& d, int64_t N, double Lx, double Ly, double sigma, double dmove, int nselect,
                uint64_t seed, int precision) {
    int mx, my;
    double wx, wy;
    const int rule = precision >> 8;   // HDMC_CELLS_SQRT2 or 0
    precision &= 0xFF;
    if (N < 1 || nselect < 1 || nselect > 255) return HDMC_EINVAL;
    if (precision != HDMC_FP64 && precision != HDMC_FP32_LOCAL) return HDMC_EINVAL;
    if (!make_grid(Lx, Ly, sigma, mx, my, wx, wy, rule)) return HDMC_EINVAL;
    if (!(dmove > 0) || !(dmove < 0.5 * wx) || !(dmove < 0.5 * wy)) return HDMC_EINVAL;
    if ((int64_t)mx * my * kSlots < N) return HDMC_EINVAL;
    if ((int64_t)mx * my >= (int64_t(1) << 32)) return HDMC_EINVAL;   // kernels index cells in 32 bits
    Geometry& g = d.g;
    g = Geometry{};
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
    g.d = dmove;
    g.df = (float)dmove;
    g.nsel = nselect;
    g.key0 = (uint32_t)seed;
    g.key1 = (uint32_t)(seed >> 32);
    g.row0 = 0;
    g.ylo = g.slo = 0;
    g.yhi = g.shi = my - 1;
    g.dense = 10 * N >= 13 * g.C;   // 1.3 disks or more per cell on average
    d.N = N;
    d.Lx = Lx;
    d.Ly = Ly;
    d.prec = precision;
    return HDMC_OK;
}

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


int bin_positions(const SysDesc& h, const double* xy, HostState& hs) {
    const Geometry& g = h.g;
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign((size_t)g.C, 0);
    for (int64_t p = 0; p < h.N; ++p) {
        const double x = xy[2 * p], y = xy[2 * p + 1];
        if (!(x >= 0.0 && x <= h.Lx && y >= 0.0 && y <= h.Ly)) return HDMC_EINVAL;
        int cx, cy;
        double lx, ly;
        bin_axis(x, g.wx, g.mx, cx, lx);
        bin_axis(y, g.wy, g.my, cy, ly);
        const int64_t c = (int64_t)cy * g.mx + cx;
        if (hs.cnt[c] >= kSlots) return HDMC_EOVERFLOW;
        const int j = hs.cnt[c]++;
        if (h.prec == HDMC_FP32_LOCAL) {
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
bool any_overlap(const SysDesc& h, const HostState& hs) {
    const Geometry& g = h.g;
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
                            if (h.prec == HDMC_FP64) {
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

// A caller's state (hdmc_get_state layout) checked and copied: counts <= 4,
// occupied coordinates in [0, w) of the precision (binary32 values for a
// binary32 system), N disks in all.  HDMC_EINVAL otherwise.
int state_from_local(const SysDesc& d, const double* local, const uint8_t* counts, HostState& hs) {
    const Geometry& g = d.g;
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign(counts, counts + g.C);
    int64_t total = 0;
    for (int64_t c = 0; c < g.C; ++c) {
        if (hs.cnt[c] > kSlots) return HDMC_EINVAL;
        total += hs.cnt[c];
        for (int j = 0; j < hs.cnt[c]; ++j) {
            const double x = local[2 * (4 * c + j)], y = local[2 * (4 * c + j) + 1];
            const bool fits = d.prec == HDMC_FP64 ? (x >= 0 && x < g.wx && y >= 0 && y < g.wy)
                                                  : ((double)(float)x == x && (double)(float)y == y && x >= 0 &&
                                                     (float)x < g.wxf && y >= 0 && (float)y < g.wyf);
            if (!fits) return HDMC_EINVAL;
            hs.loc[2 * (4 * c + j)] = x;
            hs.loc[2 * (4 * c + j) + 1] = y;
        }
    }
    return total == d.N ? HDMC_OK : HDMC_EINVAL;
}

// Canonical host state <-> set-major device cells (x0..x3 then y0..y3 per cell).
void pack(const SysDesc& h, const HostState& hs, std::vector<char>& raw) {
    const Geometry& g = h.g;
    const size_t el = h.prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    raw.assign((size_t)g.C * 8 * el, 0);
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            const long long s = storage_index(g, cx, cy);
            for (int j = 0; j < kSlots; ++j) {
                const double x = j < hs.cnt[c] ? hs.loc[2 * (4 * c + j)] : kEmpty;
                const double y = j < hs.cnt[c] ? hs.loc[2 * (4 * c + j) + 1] : kEmpty;
                if (h.prec == HDMC_FP64) {
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

void unpack(const SysDesc& h, const std::vector<char>& raw, HostState& hs) {
    const Geometry& g = h.g;
    const size_t el = h.prec == HDMC_FP64 ? sizeof(double) : sizeof(float);
    hs.loc.assign(8 * (size_t)g.C, kEmpty);
    hs.cnt.assign((size_t)g.C, 0);
    for (int cy = 0; cy < g.my; ++cy)
        for (int cx = 0; cx < g.mx; ++cx) {
            const int64_t c = (int64_t)cy * g.mx + cx;
            const long long s = storage_index(g, cx, cy);
            int n = 0;
            for (int j = 0; j < kSlots; ++j) {
                double x, y;
                if (h.prec == HDMC_FP64) {
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


int start_state(const SysDesc& d, HostState& hs) {
    int64_t nx, ny;
    if (d.N < 2 || (d.N & 1) || !lattice_shape(d.N, d.Lx, d.Ly, nx, ny)) return HDMC_EINVAL;
    std::vector<double> xy;
    lattice_positions(d.N, d.Lx, d.Ly, d.g.sigma, d.g.key0, d.g.key1, nx, ny, xy);
    int e = bin_positions(d, xy.data(), hs);
    if (!e && any_overlap(d, hs)) e = HDMC_EOVERLAP;
    return e;
}

void squared_edges(double sigma, double* E) {
    const double dr = kHistDr * sigma;
    for (int k = 0; k <= kHistBins; ++k) {
        const double edge = sigma + (double)k * dr;
        E[k] = edge * edge;
    }
}

double pressure_from_hist(const SysDesc& d, const unsigned long long* hh, int64_t ns, double* g_contact) {
    const double sigma = d.g.sigma, dr = kHistDr * sigma, c = kFitRange * sigma;
    const double rho = (double)d.N / (d.Lx * d.Ly);
    std::vector<double> t, gv;
    for (int i = 0; i < kHistBins; ++i) {
        const double r0 = sigma + dr * i, r1 = sigma + dr * (i + 1);
        const double R = (2.0 / 3.0) * (r1 * r1 * r1 - r0 * r0 * r0) / (r1 * r1 - r0 * r0);   // Eq. R
        if (!(R > sigma && R <= sigma + c)) continue;
        const double gR = (double)hh[i] / ((double)ns * (double)d.N * rho * 2.0 * M_PI * R * dr);   // Eq. gR
        t.push_back((R - sigma) / c);
        gv.push_back(gR);
    }
    const double g0 = poly_intercept(t, gv, kFitDegree);
    if (g_contact) *g_contact = g0;
    return 1.0 + 0.5 * M_PI * rho * sigma * sigma * g0;   // Eq. P
}

}  // namespace hdmc
