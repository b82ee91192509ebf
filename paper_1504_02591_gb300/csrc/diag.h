// diag.h: kernels of the paper's diagnostics that are not particle kernels.
#pragma once
#include <cuda_runtime.h>

#include "types.h"

namespace rg {

// Sec. 4.1 (Eq. irrotational): out(k) = in(k) kd_j kd_x / (k^2 N^3) on the half grid of the
// library's transform layout (M: [kx][ky][kz < N/2], Q: [kx][ky] at kz = N/2), derivative
// wavenumbers zero at the Nyquist index, zero at k = 0; the 1/N^3 of the inverse transform is
// folded in.
cudaError_t launch_helmholtz_k(const Field& in, const Field& out, int j, const Geometry& g, cudaStream_t st);
// curl_b = (j == 0 ? psi_x : 0) - grad_a over n values (Eq. solenoidal as the remainder).
cudaError_t launch_solenoidal(const float* psi_x, const float* grad_a, float* curl_b, size_t n, int j,
                              cudaStream_t st);

}  // namespace rg
