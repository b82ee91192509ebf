// conv.h: launcher of the x / y Gaussian-smoothing convolution passes.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace rg {

struct ConvArgs {
  float* f[2];           // real fields smoothed in place
  int nf;                // 1 or 2
  int n;                 // mesh side
  int axis;              // 0: along x, 1: along y
  const float* taps;     // ntap kernel values g[t0], g[t0 + 1], ...
  int ntap;              // 2K + 1, or n for a kernel that does not decay within the box
  int t0;                // first offset (-K, or -n/2)
  int count;             // count nodes of f[nf - 1] that are > 0 (partials[2 b + 1])
  double* partials;
};

int conv_blocks(int n);
size_t conv_smem(int n, int nf, int ntap);
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t st);

}  // namespace rg
