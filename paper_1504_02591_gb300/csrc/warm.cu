// warm.cu: node-wise fields for the learned warm start.  The line of sight at a node is the same
// float32 unit vector the radial-projection pass uses: node offsets from the observer (computed in
// float64 on the host) normalised with rsqrt, zero at the observer; or the fixed direction.  A
// coarse node of level l is the mean over its 2^l x 2^l x 2^l block of mesh nodes.
#include "warm.h"

namespace rg {

namespace {

__device__ __forceinline__ void node_rhat(const Geometry& g, int ix, int iy, int iz, float& rx, float& ry, float& rz) {
  if (g.los_mode == 1) {
    rx = g.los.x; ry = g.los.y; rz = g.los.z;
    return;
  }
  const int n = g.n;
  const float dx = g.off[ix], dy = g.off[n + iy], dz = g.off[2 * n + iz];
  const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float inv = q > 0.f ? rsqrtf(q) : 0.f;
  rx = dx * inv; ry = dy * inv; rz = dz * inv;
}

__global__ void features_kernel(const float* __restrict__ delta, const Geometry g, int level, float* __restrict__ feat) {
  const int n = g.n, f = 1 << level, nc = n >> level;
  const long long ncv = (long long)nc * nc * nc;
  const float w = 1.f / (float)(f * f * f);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncv; c += (long long)gridDim.x * blockDim.x) {
    const int cx = (int)(c / ((long long)nc * nc)), cy = (int)((c / nc) % nc), cz = (int)(c % nc);
    float sd = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    for (int a = 0; a < f; ++a)
      for (int b = 0; b < f; ++b) {
        const int ix = cx * f + a, iy = cy * f + b;
        const float* drow = delta + ((long long)ix * n + iy) * n + (long long)cz * f;
        for (int e = 0; e < f; ++e) {
          float rx, ry, rz;
          node_rhat(g, ix, iy, cz * f + e, rx, ry, rz);
          sd += drow[e];
          sx += rx;
          sy += ry;
          sz += rz;
        }
      }
    float* o = feat + 5 * c;
    o[0] = sd * w;
    o[1] = sx * w;
    o[2] = sy * w;
    o[3] = sz * w;
  }
}

__global__ void radial_kernel(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
                              const Geometry g, float coef, int level, float* __restrict__ out, int stride, int offset,
                              float* __restrict__ copy) {
  const int n = g.n, f = 1 << level, nc = n >> level;
  const long long ncv = (long long)nc * nc * nc;
  const float w = 1.f / (float)(f * f * f);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncv; c += (long long)gridDim.x * blockDim.x) {
    const int cx = (int)(c / ((long long)nc * nc)), cy = (int)((c / nc) % nc), cz = (int)(c % nc);
    float su = 0.f;
    for (int a = 0; a < f; ++a)
      for (int b = 0; b < f; ++b) {
        const int ix = cx * f + a, iy = cy * f + b;
        const long long v0 = ((long long)ix * n + iy) * n + (long long)cz * f;
        for (int e = 0; e < f; ++e) {
          const long long v = v0 + e;
          float u;
          if (py) {
            float rx, ry, rz;
            node_rhat(g, ix, iy, cz * f + e, rx, ry, rz);
            u = coef * fmaf(px[v], rx, fmaf(py[v], ry, pz[v] * rz));
          } else {
            u = coef * px[v];
          }
          su += u;
        }
      }
    const float r = level ? su * w : su;
    out[c * stride + offset] = r;
    if (copy) copy[c] = r;
  }
}

}  // namespace

cudaError_t launch_features(const float* delta, const Geometry& g, int level, float* feat, cudaStream_t st) {
  features_kernel<<<152 * 16, 256, 0, st>>>(delta, g, level, feat);
  return cudaGetLastError();
}

cudaError_t launch_radial(const float* px, const float* py, const float* pz, const Geometry& g, float coef, int level,
                          float* out, int stride, int offset, float* copy, cudaStream_t st) {
  radial_kernel<<<152 * 16, 256, 0, st>>>(px, py, pz, g, coef, level, out, stride, offset, copy);
  return cudaGetLastError();
}

}  // namespace rg
