// warm.h: node-wise fields for the learned warm start (network inputs, radial displacement).
#pragma once
#include <cuda_runtime.h>

#include "types.h"

namespace rg {

// feat[v][0] = delta[v], feat[v][1..3] = r(v) (line of sight at the node), channels-last, stride 5
cudaError_t launch_features(const float* delta, const Geometry& g, float* feat, cudaStream_t st);

// out[v * stride + offset] = coef * (psi_x r_x + psi_y r_y + psi_z r_z)(v)
cudaError_t launch_radial(const float* px, const float* py, const float* pz, const Geometry& g, float coef,
                          float* out, int stride, int offset, cudaStream_t st);

}  // namespace rg
