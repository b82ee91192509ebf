// fd.cu: the finite-difference configuration-space method of Sec. 2.1 (Eq. mainpot), the paper's
// comparison method, as a matrix-free operator on the GPU.
//
// A phi = grad^2 phi + beta div((grad phi . r) r) with the stencils of Sec. 2.1: the 7-point
// Laplacian over the 6 face neighbours (set A) and, for the line-of-sight term,
//   -2 phi_0 / g^2 + sum_B (x_i^2 / (g^2 r^2) +- x_i / (g r^2)) phi_(+-i)
//                  + sum_C (-1)^p x_i x_j / (2 g^2 r^2) phi_(+-i,+-j)
// (x the node's offset from the observer, r = |x|; B the face and C the edge neighbours; p = 0 when
// the two offsets share their sign).  For a fixed line of sight u the term is
// sum_ij u_i u_j d_i d_j phi with the same second differences and no 1/r term.  phi = 0 outside the
// mesh.  The solver (recon.cu) inverts A with BiCGStab preconditioned by the FFT inverse of the
// periodic 7-point Laplacian; this file holds its kernels.
#include "cic.h"
#include "fd.h"

namespace rg {

namespace {

__device__ __forceinline__ double at(const float* __restrict__ p, int n, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)n || (unsigned)y >= (unsigned)n || (unsigned)z >= (unsigned)n) return 0.0;
  return (double)__ldg(p + ((size_t)x * n + y) * n + z);
}

__global__ void __launch_bounds__(256) fd_apply_kernel(const float* __restrict__ phi, float* __restrict__ out,
                                                       FDArgs a) {
  const int n = a.n;
  const size_t total = (size_t)n * n * n;
  const double ig2 = 1.0 / (a.g * a.g), ig = 1.0 / a.g;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e / ((size_t)n * n)), y = (int)((e / n) % n), z = (int)(e % n);
    const int c[3] = {x, y, z};
    const double p0 = at(phi, n, x, y, z);
    double face[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int q[3] = {c[0], c[1], c[2]};
        q[d] += s ? -1 : 1;
        face[d][s] = at(phi, n, q[0], q[1], q[2]);
      }
    double lap = -6.0 * p0;
#pragma unroll
    for (int d = 0; d < 3; ++d) lap += face[d][0] + face[d][1];
    double acc = lap * ig2;
    if (a.beta != 0.0) {
      double xs[3], inv_r2, first;
      if (a.los_mode == 1) {
        xs[0] = a.los.x;
        xs[1] = a.los.y;
        xs[2] = a.los.z;
        inv_r2 = 1.0;
        first = 0.0;
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) xs[d] = (double)a.off[d * n + c[d]];
        const double r2 = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
        inv_r2 = r2 > 0.0 ? 1.0 / r2 : 0.0;
        first = 1.0;
      }
      double rsd = inv_r2 > 0.0 ? -2.0 * p0 * ig2 : 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double c2 = xs[d] * xs[d] * inv_r2 * ig2, c1 = first * xs[d] * inv_r2 * ig;
        rsd += (c2 + c1) * face[d][0] + (c2 - c1) * face[d][1];
      }
#pragma unroll
      for (int d0 = 0; d0 < 3; ++d0)
#pragma unroll
        for (int d1 = d0 + 1; d1 < 3; ++d1) {
          const double cc = xs[d0] * xs[d1] * inv_r2 * 0.5 * ig2;
#pragma unroll
          for (int s0 = 0; s0 < 2; ++s0)
#pragma unroll
            for (int s1 = 0; s1 < 2; ++s1) {
              int q[3] = {c[0], c[1], c[2]};
              q[d0] += s0 ? -1 : 1;
              q[d1] += s1 ? -1 : 1;
              rsd += (s0 == s1 ? cc : -cc) * at(phi, n, q[0], q[1], q[2]);
            }
        }
      acc += a.beta * rsd;
    }
    out[e] = (float)acc;
  }
}

__global__ void __launch_bounds__(256) fd_gradient_kernel(const float* __restrict__ phi, float* __restrict__ psi,
                                                          FDArgs a) {
  const int n = a.n;
  const size_t total = (size_t)n * n * n;
  const double h = 0.5 / a.g;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e / ((size_t)n * n)), y = (int)((e / n) % n), z = (int)(e % n);
    psi[e] = (float)(-(at(phi, n, x + 1, y, z) - at(phi, n, x - 1, y, z)) * h);
    psi[total + e] = (float)(-(at(phi, n, x, y + 1, z) - at(phi, n, x, y - 1, z)) * h);
    psi[2 * total + e] = (float)(-(at(phi, n, x, y, z + 1) - at(phi, n, x, y, z - 1)) * h);
  }
}

__global__ void __launch_bounds__(256) fd_precond_kernel(const Field f, int n, double L) {
  const int h = n / 2;
  const size_t nm = (size_t)n * n * h, nq = (size_t)n * n;
  const double g = L / n, n3 = (double)n * n * n;
  const double k0 = -L * L / (3.0 * M_PI * M_PI) / n3;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nm + nq; e += (size_t)gridDim.x * blockDim.x) {
    int kx, ky, kz;
    if (e < nm) {
      kx = (int)(e / ((size_t)n * h));
      ky = (int)((e / h) % n);
      kz = (int)(e % h);
    } else {
      kx = (int)((e - nm) / n);
      ky = (int)((e - nm) % n);
      kz = h;
    }
    // 2 cos(2 pi m / N) - 2 per axis (the sign of m does not matter)
    const double lam = (2.0 * cospi(2.0 * kx / n) - 2.0 + 2.0 * cospi(2.0 * ky / n) - 2.0 +
                        2.0 * cospi(2.0 * kz / n) - 2.0) / (g * g);
    const float fac = (float)((kx | ky | kz) == 0 ? k0 : 1.0 / (lam * n3));
    float2* v = e < nm ? f.M + e : f.Q + (e - nm);
    *v = make_float2(v->x * fac, v->y * fac);
  }
}

__global__ void __launch_bounds__(256) dot_kernel(const float* __restrict__ x, const float* __restrict__ y, size_t n,
                                                  double* __restrict__ partials) {
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += (double)x[i] * (double)y[i];
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    partials[blockIdx.x] = r;
  }
}

__global__ void fd_dir_kernel(float* __restrict__ y, const float* __restrict__ x, const float* __restrict__ z,
                              double a, double b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)((double)x[i] + a * ((double)y[i] - b * (double)z[i]));
}

__global__ void fd_sub_kernel(float* __restrict__ y, const float* __restrict__ x, const float* __restrict__ z,
                              double a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)((double)x[i] - a * (double)z[i]);
}

__global__ void fd_acc_kernel(float* __restrict__ y, const float* __restrict__ x, const float* __restrict__ z,
                              double a, double b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)((double)y[i] + a * (double)x[i] + b * (double)z[i]);
}

constexpr int kGrid = 152 * 8;

}  // namespace

cudaError_t launch_fd_apply(const float* phi, float* out, const FDArgs& a, cudaStream_t st) {
  fd_apply_kernel<<<kGrid, 256, 0, st>>>(phi, out, a);
  return cudaGetLastError();
}

cudaError_t launch_fd_gradient(const float* phi, float* psi, const FDArgs& a, cudaStream_t st) {
  fd_gradient_kernel<<<kGrid, 256, 0, st>>>(phi, psi, a);
  return cudaGetLastError();
}

cudaError_t launch_fd_precond_k(const Field& f, int n, double L, cudaStream_t st) {
  fd_precond_kernel<<<kGrid, 256, 0, st>>>(f, n, L);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float* x, const float* y, size_t n, double* partials, int blocks, cudaStream_t st) {
  dot_kernel<<<blocks, 256, 0, st>>>(x, y, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_fd_dir(float* y, const float* x, const float* z, double a, double b, size_t n, cudaStream_t st) {
  fd_dir_kernel<<<kGrid, 256, 0, st>>>(y, x, z, a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_fd_sub(float* y, const float* x, const float* z, double a, size_t n, cudaStream_t st) {
  fd_sub_kernel<<<kGrid, 256, 0, st>>>(y, x, z, a, n);
  return cudaGetLastError();
}

cudaError_t launch_fd_acc(float* y, const float* x, const float* z, double a, double b, size_t n, cudaStream_t st) {
  fd_acc_kernel<<<kGrid, 256, 0, st>>>(y, x, z, a, b, n);
  return cudaGetLastError();
}

}  // namespace rg
