// diag.cu: the plane-parallel Helmholtz split of Sec. 4.1 (Eq. Helmholtz): (Psi.x) x = grad A +
// curl B with grad A_j(k) = (k_j k_x / k^2) Psi_x(k) (Eq. irrotational) and curl B the remainder
// (Eq. solenoidal).  The transforms are the library's own FFT passes; this file holds the
// pointwise Fourier-space product and the remainder.
#include "diag.h"

namespace rg {

__global__ void __launch_bounds__(256) helmholtz_k_kernel(const Field in, const Field out, int j, Geometry g) {
  const int n = g.n, h = n / 2;
  const size_t nm = (size_t)n * n * h, nq = (size_t)n * n;
  const float inv_n3 = g.inv_n3;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nm + nq; e += (size_t)gridDim.x * blockDim.x) {
    int kx, ky, kz;
    if (e < nm) {
      kx = (int)(e / ((size_t)n * h));
      ky = (int)((e / h) % n);
      kz = (int)(e % h);
    } else {
      const size_t q = e - nm;
      kx = (int)(q / n);
      ky = (int)(q % n);
      kz = h;
    }
    const int mx = kx < h ? kx : kx - n, my = ky < h ? ky : ky - n;
    const float fx = g.kf * mx, fy = g.kf * my, fz = g.kf * kz;
    const float k2 = fx * fx + fy * fy + fz * fz;
    const float dx = kx == h ? 0.f : fx, dy = ky == h ? 0.f : fy, dz = kz == h ? 0.f : fz;
    const float dj = j == 0 ? dx : (j == 1 ? dy : dz);
    const float fac = k2 > 0.f ? dj * dx / k2 * inv_n3 : 0.f;
    const float2 v = e < nm ? in.M[e] : in.Q[e - nm];
    const float2 r = make_float2(v.x * fac, v.y * fac);
    if (e < nm) out.M[e] = r;
    else out.Q[e - nm] = r;
  }
}

__global__ void __launch_bounds__(256) solenoidal_kernel(const float* __restrict__ psi_x, const float* __restrict__ ga,
                                                         float* __restrict__ cb, size_t n, int j) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    cb[i] = (j == 0 ? psi_x[i] : 0.f) - ga[i];
}

cudaError_t launch_helmholtz_k(const Field& in, const Field& out, int j, const Geometry& g, cudaStream_t st) {
  helmholtz_k_kernel<<<152 * 8, 256, 0, st>>>(in, out, j, g);
  return cudaGetLastError();
}

cudaError_t launch_solenoidal(const float* psi_x, const float* grad_a, float* curl_b, size_t n, int j,
                              cudaStream_t st) {
  solenoidal_kernel<<<152 * 8, 256, 0, st>>>(psi_x, grad_a, curl_b, n, j);
  return cudaGetLastError();
}

}  // namespace rg
