// cic.h: launchers of the particle kernels and the reduction helpers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace rg {

struct ShiftArgs {
  const float* psi[3];   // real Psi components, N^3 each
  int n;
  double scale;          // N / L
  double L;
  int is_galaxy;
  float f;               // growth rate of the galaxy RSD term
  int los_mode;          // 0 radial, 1 fixed
  float3 los;            // fixed LOS unit vector
  const float* off;      // 3 N node offsets from the observer, per axis (radial)
  float H;               // cell size: a particle's offset is off[node] + t H, its image in [0, L)
  int periodic;
  float* shift;          // (n, 3) out
  double* pos_out;       // (n, 3) out or null
};

constexpr int kDepositBlocks = 152 * 8;

// CIC (or, with ngp, nearest-grid-point) deposit; the weight sum of each block into partials.
cudaError_t launch_deposit(const void* pos, int dtype, const float* w, long long np, int n, double L,
                           float* rho, double* partials, int blocks, cudaStream_t st, int ngp = 0);
// Counts of particles in nbins equal radial shells [rmin, rmax) about obs (counts zeroed by the caller).
cudaError_t launch_radial_hist(const void* pos, int dtype, long long np, double3 obs, double rmin, double rmax,
                               int nbins, unsigned long long* counts, cudaStream_t st);
// FKP weights 1 / (1 + nbar P0) with nbar (device, nbins) of each particle's shell, 0 outside.
cudaError_t launch_fkp(const void* pos, int dtype, long long np, double3 obs, double rmin, double rmax, int nbins,
                       const double* nbar, double P0, float* w, cudaStream_t st);
cudaError_t launch_shift(const void* pos, int dtype, long long np, const ShiftArgs& a, cudaStream_t st);
// red[dst + q] (=|+=) the sum over b < nblocks of partials[b nq + q], q < nq <= 4, in a fixed order.
// bsum (kFinalizeBlocks x 4 doubles) and counter (zeroed; left zeroed) let several blocks share the
// sum; with nulls one block does it.
constexpr int kFinalizeBlocks = 64;
cudaError_t launch_finalize(const double* partials, int nblocks, int nq, double* red, int dst, int accumulate,
                            cudaStream_t st, double* bsum = nullptr, unsigned int* counter = nullptr);
cudaError_t launch_add_scalar(float* x, size_t n, float v, cudaStream_t st);

// Ratio statistics of the paper's diagnostics (Eq. ratio; Tables 1-3): per block, the number of
// ratios num/den inside [lo, hi] (a zero denominator is outside), their sum and sum of squares in
// float64, and the number of points: partials[4 b + 0..3].
struct RatioArgs {
  const float* num[3];   // radial form: the two vector fields (Psi_real, Psi_est), N^3 each
  const float* den[3];
  int n;
  double scale;          // N / L
  int los_mode;
  float3 los;
  const float* off;      // 3 N node offsets from the observer
  float H;
  double lo, hi;
  double* partials;
};
// (Psi_num . r)/(Psi_den . r) at each particle, both fields CIC-interpolated, r the particle's line
// of sight (its image in [0, L), as in the shift).
cudaError_t launch_radial_ratio(const void* pos, int dtype, long long np, const RatioArgs& a, int blocks,
                                cudaStream_t st);
// num[i] / den[i] over n values.
cudaError_t launch_ratio(const float* num, const float* den, size_t n, double lo, double hi, double* partials,
                         int blocks, cudaStream_t st);

}  // namespace rg
