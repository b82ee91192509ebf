// fd.h: kernels of the finite-difference configuration-space method (Sec. 2.1, Eq. mainpot).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "types.h"

namespace rg {

struct FDArgs {
  int n;
  double g;              // mesh spacing L / N
  double beta;           // coefficient of the line-of-sight term (f / b)
  int los_mode;          // 0 radial, 1 fixed
  double3 los;           // fixed line of sight (unit)
  const float* off;      // 3 N node offsets from the observer (radial)
};

// out = A phi: the 7-point Laplacian plus beta times the line-of-sight stencil of Sec. 2.1, phi = 0
// outside the mesh; sums in float64.
cudaError_t launch_fd_apply(const float* phi, float* out, const FDArgs& a, cudaStream_t st);
// Psi_j = -(phi(+j) - phi(-j)) / (2 g), phi = 0 outside the mesh; psi holds 3 N^3 values.
cudaError_t launch_fd_gradient(const float* phi, float* psi, const FDArgs& a, cudaStream_t st);
// The preconditioner's Fourier-space factor on the library's half grid (M: [kx][ky][kz < N/2],
// Q: kz = N/2): 1 / (N^3 lambda(k)), lambda the periodic 7-point Laplacian's eigenvalue
// sum_i (2 cos(k_i g) - 2) / g^2, and -L^2 / (3 pi^2 N^3) at k = 0.
cudaError_t launch_fd_precond_k(const Field& f, int n, double L, cudaStream_t st);
// Per-block float64 partial sums of x . y (partials[b]), for the Krylov solver's inner products.
cudaError_t launch_dot(const float* x, const float* y, size_t n, double* partials, int blocks, cudaStream_t st);
// y = x + a (y - b z)  (BiCGStab's search direction: p = r + beta (p - omega v))
cudaError_t launch_fd_dir(float* y, const float* x, const float* z, double a, double b, size_t n, cudaStream_t st);
// y = x - a z
cudaError_t launch_fd_sub(float* y, const float* x, const float* z, double a, size_t n, cudaStream_t st);
// y += a x + b z
cudaError_t launch_fd_acc(float* y, const float* x, const float* z, double a, double b, size_t n, cudaStream_t st);

}  // namespace rg
