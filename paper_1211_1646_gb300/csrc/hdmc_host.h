// hdmc_host.h -- host-side helpers shared by the C entry points (see
// hdmc_host.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "hdmc.h"
#include "hdmc_device.cuh"

namespace hdmc {

// One system: geometry, number of disks, box and coordinate precision.
struct SysDesc {
    Geometry g;
    int64_t N;
    double Lx, Ly;
    int prec;
    size_t coord_bytes() const { return prec == HDMC_FP64 ? sizeof(double) : sizeof(float); }
    size_t cells_bytes() const { return (size_t)g.C * 8 * coord_bytes(); }
};

// Canonical host copy of a state: loc[(4c+j)*2+k], cnt[c], c = cy*mx + cx.
struct HostState {
    std::vector<double> loc;
    std::vector<uint8_t> cnt;
};

int cuda_code(cudaError_t e);
int error_code(unsigned int device_error);   // device error word -> HDMC_E* (0: HDMC_OK)
bool make_grid(double Lx, double Ly, double sigma, int& mx, int& my, double& wx, double& wy, int rule = 0);
// precision: HDMC_FP64 or HDMC_FP32_LOCAL, optionally | HDMC_CELLS_SQRT2 (d.prec is the bare precision)
int make_system(SysDesc& d, int64_t N, double Lx, double Ly, double sigma, double dmove, int nselect,
                uint64_t seed, int precision);
bool lattice_shape(int64_t N, double Lx, double Ly, int64_t& nx, int64_t& ny);
void lattice_positions(int64_t N, double Lx, double Ly, double sigma, uint32_t k0, uint32_t k1, int64_t nx,
                       int64_t ny, std::vector<double>& xy);
int bin_positions(const SysDesc& d, const double* xy, HostState& hs);
bool any_overlap(const SysDesc& d, const HostState& hs);
int start_state(const SysDesc& d, HostState& hs);   // hexagonal start, binned and checked
int state_from_local(const SysDesc& d, const double* local, const uint8_t* counts, HostState& hs);
void pack(const SysDesc& d, const HostState& hs, std::vector<char>& raw);
void unpack(const SysDesc& d, const std::vector<char>& raw, HostState& hs);
void squared_edges(double sigma, double* E);          // kHistBins + 1 values
double poly_intercept(const std::vector<double>& t, const std::vector<double>& y, int deg);
double pressure_from_hist(const SysDesc& d, const unsigned long long* hist, int64_t n_samples, double* g_contact);

}  // namespace hdmc
