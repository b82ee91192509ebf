// warm.h: node-wise fields for the learned warm start (network inputs, radial displacement), on
// the mesh (level 0) or averaged over blocks of 2^level x 2^level x 2^level nodes.
#pragma once
#include <cuda_runtime.h>

#include "types.h"

namespace rg {

// feat[c][0] = mean of delta over the block of coarse node c, feat[c][1..3] = mean of the line of
// sight r over the block; channels-last with stride 5 on the (N >> level)^3 grid.
cudaError_t launch_features(const float* delta, const Geometry& g, int level, float* feat, cudaStream_t st);

// out[c * stride + offset] (and copy[c] when not null) = block mean of coef * (p . r) when py and pz
// are given, else of coef * px.
cudaError_t launch_radial(const float* px, const float* py, const float* pz, const Geometry& g, float coef,
                          int level, float* out, int stride, int offset, float* copy, cudaStream_t st);

}  // namespace rg
