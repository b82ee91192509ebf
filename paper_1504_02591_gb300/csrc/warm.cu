// warm.cu: node-wise fields for the learned warm start.  The line of sight at a node is the same
// float32 unit vector the radial-projection pass uses: node offsets from the observer (computed in
// float64 on the host) normalised with rsqrt, zero at the observer; or the fixed direction.
#include "warm.h"

namespace rg {

namespace {

__device__ __forceinline__ void node_rhat(const Geometry& g, long long v, float& rx, float& ry, float& rz) {
  const int n = g.n;
  if (g.los_mode == 1) {
    rx = g.los.x; ry = g.los.y; rz = g.los.z;
    return;
  }
  const int ix = (int)(v / ((long long)n * n)), iy = (int)((v / n) % n), iz = (int)(v % n);
  const float dx = g.off[ix], dy = g.off[n + iy], dz = g.off[2 * n + iz];
  const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float inv = q > 0.f ? rsqrtf(q) : 0.f;
  rx = dx * inv; ry = dy * inv; rz = dz * inv;
}

__global__ void features_kernel(const float* __restrict__ delta, const Geometry g, float* __restrict__ feat) {
  const long long nv = (long long)g.n * g.n * g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    float rx, ry, rz;
    node_rhat(g, v, rx, ry, rz);
    float* f = feat + 5 * v;
    f[0] = delta[v];
    f[1] = rx;
    f[2] = ry;
    f[3] = rz;
  }
}

__global__ void radial_kernel(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
                              const Geometry g, float coef, float* __restrict__ out, int stride, int offset) {
  const long long nv = (long long)g.n * g.n * g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    float rx, ry, rz;
    node_rhat(g, v, rx, ry, rz);
    out[v * stride + offset] = coef * fmaf(px[v], rx, fmaf(py[v], ry, pz[v] * rz));
  }
}

}  // namespace

cudaError_t launch_features(const float* delta, const Geometry& g, float* feat, cudaStream_t st) {
  features_kernel<<<152 * 16, 256, 0, st>>>(delta, g, feat);
  return cudaGetLastError();
}

cudaError_t launch_radial(const float* px, const float* py, const float* pz, const Geometry& g, float coef,
                          float* out, int stride, int offset, cudaStream_t st) {
  radial_kernel<<<152 * 16, 256, 0, st>>>(px, py, pz, g, coef, out, stride, offset);
  return cudaGetLastError();
}

}  // namespace rg
