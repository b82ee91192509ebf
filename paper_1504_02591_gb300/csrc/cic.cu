// cic.cu: cloud-in-cell mass assignment and interpolation, the reconstruction shift, reductions.
//
// Mass assignment (Sec. 3 bins tracers on the mesh; this library uses CIC instead of NGP): a
// particle at grid coordinate u = x N / L deposits w (1 - t) and w t on the nodes floor(u) and
// floor(u) + 1 of each axis, t = u - floor(u), with periodic wrap.  The same kernel interpolates
// Psi back to particles for the shift of Sec. 1 (reversing Eq. Lagrange x = q + Psi).
#include <mutex>

#include "../../include/recon.h"
#include "cic.h"

namespace rg {

// Nodes and weights of one particle.  u 2^32 = x times scale 2^32 (exact scaling: the same rounding
// as u), rounded down to an integer T: floor(u) = T >> 32 and t = (T mod 2^32) 2^-32.  Two float64
// operations per axis (float64 runs at a small fraction of the float32 rate on this GPU).
template <typename PT>
__device__ __forceinline__ void cic_setup(const PT* __restrict__ pos, long long p, int n, double scale,
                                          int (&i0)[3], int (&i1)[3], float (&t)[3]) {
  const double scale32 = scale * 4294967296.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long T = __double2ll_rd((double)pos[3 * p + a] * scale32);
    t[a] = (float)(uint32_t)T * 2.3283064365386963e-10f;   // 2^-32
    int c = (int)(T >> 32);
    if (c < 0 || c >= n) c = ((c % n) + n) % n;   // outside [0, L): periodic image
    i0[a] = c;
    i1[a] = (c + 1 == n) ? 0 : c + 1;
  }
}

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

template <typename PT>
__global__ void __launch_bounds__(256) deposit_kernel(const PT* __restrict__ pos, const float* __restrict__ w,
                                                      long long np, int n, double scale,
                                                      float* __restrict__ rho, double* __restrict__ partials) {
  double wsum = 0.0;
  const size_t nn = (size_t)n;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    float t[3];
    cic_setup(pos, p, n, scale, i0, i1, t);
    const float wp = w ? w[p] : 1.f;
    wsum += wp;
    const float wx0 = wp * (1.f - t[0]), wx1 = wp * t[0];
    const float wy0 = 1.f - t[1], wy1 = t[1];
    const float wz0 = 1.f - t[2], wz1 = t[2];
    const size_t r00 = ((size_t)i0[0] * nn + i0[1]) * nn, r01 = ((size_t)i0[0] * nn + i1[1]) * nn;
    const size_t r10 = ((size_t)i1[0] * nn + i0[1]) * nn, r11 = ((size_t)i1[0] * nn + i1[1]) * nn;
    atomicAdd(rho + r00 + i0[2], wx0 * wy0 * wz0);
    atomicAdd(rho + r00 + i1[2], wx0 * wy0 * wz1);
    atomicAdd(rho + r01 + i0[2], wx0 * wy1 * wz0);
    atomicAdd(rho + r01 + i1[2], wx0 * wy1 * wz1);
    atomicAdd(rho + r10 + i0[2], wx1 * wy0 * wz0);
    atomicAdd(rho + r10 + i1[2], wx1 * wy0 * wz1);
    atomicAdd(rho + r11 + i0[2], wx1 * wy1 * wz0);
    atomicAdd(rho + r11 + i1[2], wx1 * wy1 * wz1);
  }
  const double s = block_sum_d(wsum);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Nearest-grid-point binning (Sec. 3, the paper's scheme): node floor(u + 1/2) per axis, from the
// same 32.32 fixed-point coordinate as the CIC kernel (u 2^32 + 2^31 rounded down).
template <typename PT>
__global__ void __launch_bounds__(256) ngp_deposit_kernel(const PT* __restrict__ pos, const float* __restrict__ w,
                                                          long long np, int n, double scale,
                                                          float* __restrict__ rho, double* __restrict__ partials) {
  double wsum = 0.0;
  const size_t nn = (size_t)n;
  const double scale32 = scale * 4294967296.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long T = __double2ll_rd(fma((double)pos[3 * p + a], scale32, 2147483648.0));
      int k = (int)(T >> 32);
      if (k < 0 || k >= n) k = ((k % n) + n) % n;
      c[a] = k;
    }
    const float wp = w ? w[p] : 1.f;
    wsum += wp;
    atomicAdd(rho + ((size_t)c[0] * nn + c[1]) * nn + c[2], wp);
  }
  const double s = block_sum_d(wsum);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Radial number density (Sec. 3.2 n(z), in comoving distance from the observer): counts of the
// particles in nbins equal shells of [rmin, rmax), float64 distances.
template <typename PT>
__global__ void __launch_bounds__(256) radial_hist_kernel(const PT* __restrict__ pos, long long np, double3 obs,
                                                          double rmin, double inv_dr, int nbins,
                                                          unsigned long long* __restrict__ counts) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    const double dx = (double)pos[3 * p] - obs.x, dy = (double)pos[3 * p + 1] - obs.y, dz = (double)pos[3 * p + 2] - obs.z;
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double b = floor((r - rmin) * inv_dr);
    if (b >= 0.0 && b < (double)nbins) atomicAdd(counts + (int)b, 1ull);
  }
}

// FKP weights w = 1 / (1 + nbar(r) P0) (Sec. 3.2), nbar of the particle's shell, 0 outside.
template <typename PT>
__global__ void __launch_bounds__(256) fkp_kernel(const PT* __restrict__ pos, long long np, double3 obs, double rmin,
                                                  double inv_dr, int nbins, const double* __restrict__ nbar,
                                                  double P0, float* __restrict__ w) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    const double dx = (double)pos[3 * p] - obs.x, dy = (double)pos[3 * p + 1] - obs.y, dz = (double)pos[3 * p + 2] - obs.z;
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double b = floor((r - rmin) * inv_dr);
    const double nb = (b >= 0.0 && b < (double)nbins) ? nbar[(int)b] : 0.0;
    w[p] = (float)(1.0 / (1.0 + nb * P0));
  }
}

template <typename PT>
__global__ void __launch_bounds__(256) shift_kernel(const PT* __restrict__ pos, long long np, ShiftArgs a) {
  const size_t nn = (size_t)a.n;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    float t[3];
    cic_setup(pos, p, a.n, a.scale, i0, i1, t);
    const size_t r00 = ((size_t)i0[0] * nn + i0[1]) * nn, r01 = ((size_t)i0[0] * nn + i1[1]) * nn;
    const size_t r10 = ((size_t)i1[0] * nn + i0[1]) * nn, r11 = ((size_t)i1[0] * nn + i1[1]) * nn;
    const float wx0 = 1.f - t[0], wx1 = t[0], wy0 = 1.f - t[1], wy1 = t[1], wz0 = 1.f - t[2], wz1 = t[2];
    const size_t idx[8] = {r00 + i0[2], r00 + i1[2], r01 + i0[2], r01 + i1[2],
                           r10 + i0[2], r10 + i1[2], r11 + i0[2], r11 + i1[2]};
    const float cw[8] = {wx0 * wy0 * wz0, wx0 * wy0 * wz1, wx0 * wy1 * wz0, wx0 * wy1 * wz1,
                         wx1 * wy0 * wz0, wx1 * wy0 * wz1, wx1 * wy1 * wz0, wx1 * wy1 * wz1};
    float ps[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) acc = fmaf(cw[k], __ldg(a.psi[c] + idx[k]), acc);
      ps[c] = acc;
    }
    const double x0 = (double)pos[3 * p], x1 = (double)pos[3 * p + 1], x2 = (double)pos[3 * p + 2];
    float d[3];
    if (a.is_galaxy) {
      float rx, ry, rz;
      if (a.los_mode == 1) {
        rx = a.los.x; ry = a.los.y; rz = a.los.z;
      } else {
        // offset of the particle's image in [0, L) from the observer, as the brick-sorted path forms it
        const int n = a.n;
        const float dx = fmaf(t[0], a.H, a.off[i0[0]]), dy = fmaf(t[1], a.H, a.off[n + i0[1]]),
                    dz = fmaf(t[2], a.H, a.off[2 * n + i0[2]]);
        const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float ir = q > 0.f ? rsqrtf(q) : 0.f;
        rx = dx * ir; ry = dy * ir; rz = dz * ir;
      }
      const float u = a.f * fmaf(ps[0], rx, fmaf(ps[1], ry, ps[2] * rz));
      d[0] = -fmaf(u, rx, ps[0]);
      d[1] = -fmaf(u, ry, ps[1]);
      d[2] = -fmaf(u, rz, ps[2]);
    } else {
      d[0] = -ps[0]; d[1] = -ps[1]; d[2] = -ps[2];
    }
    a.shift[3 * p + 0] = d[0];
    a.shift[3 * p + 1] = d[1];
    a.shift[3 * p + 2] = d[2];
    if (a.pos_out) {
      double y[3] = {x0 + d[0], x1 + d[1], x2 + d[2]};
      if (a.periodic) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          y[c] = y[c] - floor(y[c] / a.L) * a.L;
          if (y[c] >= a.L) y[c] -= a.L;
        }
      }
      a.pos_out[3 * p + 0] = y[0];
      a.pos_out[3 * p + 1] = y[1];
      a.pos_out[3 * p + 2] = y[2];
    }
  }
}

// Sum nq interleaved partial columns: red[dst + q] (=|+=) sum_b partials[b * nq + q].
// Sums the per-block partials (nq <= 4 quantities, interleaved) in a fixed order.  With scratch
// (kFinalizeBlocks x 4 doubles and a zeroed counter), gridDim.x blocks each sum a contiguous range
// and the last block to finish adds the block sums in block order and resets the counter: float64
// adds run at a few per clock on one SM, so one block summing tens of thousands of partials takes
// tens of microseconds.  Without scratch, one block sums everything.
constexpr int kFinalizeThreads = 1024;
__global__ void __launch_bounds__(kFinalizeThreads) finalize_kernel(const double* __restrict__ partials, int nblocks,
                                                                    int nq, double* __restrict__ red, int dst,
                                                                    int accumulate, double* __restrict__ bsum,
                                                                    unsigned int* __restrict__ counter) {
  const int per = (nblocks + gridDim.x - 1) / gridDim.x;
  const int b0 = blockIdx.x * per, b1 = min(nblocks, b0 + per);
  double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) s[q] += partials[(size_t)b * nq + q];
  double t[4];
  for (int q = 0; q < nq; ++q) t[q] = block_sum_d(s[q]);
  if (gridDim.x == 1) {
    if (threadIdx.x == 0)
      for (int q = 0; q < nq; ++q) red[dst + q] = accumulate ? red[dst + q] + t[q] : t[q];
    return;
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nq; ++q) bsum[4 * blockIdx.x + q] = t[q];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* vb = bsum;
    for (int q = 0; q < nq; ++q) {
      double r = 0.0;
      for (int g = 0; g < (int)gridDim.x; ++g) r += vb[4 * g + q];
      red[dst + q] = accumulate ? red[dst + q] + r : r;
    }
    *counter = 0u;
  }
}

__global__ void add_scalar_kernel(float* __restrict__ x, size_t n, float v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += v;
}

cudaError_t launch_deposit(const void* pos, int dtype, const float* w, long long np, int n, double L,
                           float* rho, double* partials, int blocks, cudaStream_t st, int ngp) {
  if (np <= 0) return cudaSuccess;
  const double scale = (double)n / L;
  if (ngp) {
    if (dtype == 0)
      ngp_deposit_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, w, np, n, scale, rho, partials);
    else
      ngp_deposit_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, w, np, n, scale, rho, partials);
    return cudaGetLastError();
  }
  if (dtype == 0)
    deposit_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, w, np, n, scale, rho, partials);
  else
    deposit_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, w, np, n, scale, rho, partials);
  return cudaGetLastError();
}

cudaError_t launch_shift(const void* pos, int dtype, long long np, const ShiftArgs& a, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  long long want = (np + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  if (dtype == 0)
    shift_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, np, a);
  else
    shift_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, np, a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, int nq, double* red, int dst, int accumulate,
                            cudaStream_t st, double* bsum, unsigned int* counter) {
  if (nq < 1 || nq > 4) return cudaErrorInvalidValue;
  int blocks = 1;
  if (bsum && counter) {   // about 1024 partials per block, at most kFinalizeBlocks blocks
    blocks = (nblocks + 1023) / 1024;
    blocks = blocks < 1 ? 1 : (blocks > kFinalizeBlocks ? kFinalizeBlocks : blocks);
  }
  finalize_kernel<<<blocks, kFinalizeThreads, 0, st>>>(partials, nblocks, nq, red, dst, accumulate, bsum, counter);
  return cudaGetLastError();
}

cudaError_t launch_add_scalar(float* x, size_t n, float v, cudaStream_t st) {
  add_scalar_kernel<<<152 * 8, 256, 0, st>>>(x, n, v);
  return cudaGetLastError();
}

// One ratio into the running statistics (float64; the decision at the cut is taken in float64 on
// the float32 inputs).
__device__ __forceinline__ void ratio_acc(float num, float den, double lo, double hi, double (&acc)[4]) {
  acc[3] += 1.0;
  if (den != 0.f) {
    const double r = (double)num / (double)den;
    if (r >= lo && r <= hi) {
      acc[0] += 1.0;
      acc[1] += r;
      acc[2] += r * r;
    }
  }
}

__device__ __forceinline__ void ratio_flush(double (&acc)[4], double* partials) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double s = block_sum_d(acc[q]);
    if (threadIdx.x == 0) partials[4 * blockIdx.x + q] = s;
  }
}

template <typename PT>
__global__ void __launch_bounds__(256) radial_ratio_kernel(const PT* __restrict__ pos, long long np, RatioArgs a) {
  const size_t nn = (size_t)a.n;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    float t[3];
    cic_setup(pos, p, a.n, a.scale, i0, i1, t);
    const size_t r00 = ((size_t)i0[0] * nn + i0[1]) * nn, r01 = ((size_t)i0[0] * nn + i1[1]) * nn;
    const size_t r10 = ((size_t)i1[0] * nn + i0[1]) * nn, r11 = ((size_t)i1[0] * nn + i1[1]) * nn;
    const float wx0 = 1.f - t[0], wx1 = t[0], wy0 = 1.f - t[1], wy1 = t[1], wz0 = 1.f - t[2], wz1 = t[2];
    const size_t idx[8] = {r00 + i0[2], r00 + i1[2], r01 + i0[2], r01 + i1[2],
                           r10 + i0[2], r10 + i1[2], r11 + i0[2], r11 + i1[2]};
    const float cw[8] = {wx0 * wy0 * wz0, wx0 * wy0 * wz1, wx0 * wy1 * wz0, wx0 * wy1 * wz1,
                         wx1 * wy0 * wz0, wx1 * wy0 * wz1, wx1 * wy1 * wz0, wx1 * wy1 * wz1};
    float rv[3];
    if (a.los_mode == 1) {
      rv[0] = a.los.x; rv[1] = a.los.y; rv[2] = a.los.z;
    } else {
      const int n = a.n;
      const float dx = fmaf(t[0], a.H, a.off[i0[0]]), dy = fmaf(t[1], a.H, a.off[n + i0[1]]),
                  dz = fmaf(t[2], a.H, a.off[2 * n + i0[2]]);
      const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float ir = q > 0.f ? rsqrtf(q) : 0.f;
      rv[0] = dx * ir; rv[1] = dy * ir; rv[2] = dz * ir;
    }
    float un = 0.f, ud = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float gn = 0.f, gd = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gn = fmaf(cw[k], __ldg(a.num[c] + idx[k]), gn);
        gd = fmaf(cw[k], __ldg(a.den[c] + idx[k]), gd);
      }
      un = fmaf(gn, rv[c], un);
      ud = fmaf(gd, rv[c], ud);
    }
    ratio_acc(un, ud, a.lo, a.hi, acc);
  }
  ratio_flush(acc, a.partials);
}

__global__ void __launch_bounds__(256) ratio_kernel(const float* __restrict__ num, const float* __restrict__ den,
                                                    size_t n, double lo, double hi, double* __restrict__ partials) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    ratio_acc(num[i], den[i], lo, hi, acc);
  ratio_flush(acc, partials);
}

cudaError_t launch_radial_ratio(const void* pos, int dtype, long long np, const RatioArgs& a, int blocks,
                                cudaStream_t st) {
  if (dtype == 0)
    radial_ratio_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, np, a);
  else
    radial_ratio_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, np, a);
  return cudaGetLastError();
}

cudaError_t launch_radial_hist(const void* pos, int dtype, long long np, double3 obs, double rmin, double rmax,
                               int nbins, unsigned long long* counts, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  const double inv_dr = nbins / (rmax - rmin);
  const int blocks = (int)((np + 255) / 256 < 152 * 16 ? (np + 255) / 256 : 152 * 16);
  if (dtype == 0)
    radial_hist_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, np, obs, rmin, inv_dr, nbins, counts);
  else
    radial_hist_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, np, obs, rmin, inv_dr, nbins, counts);
  return cudaGetLastError();
}

cudaError_t launch_fkp(const void* pos, int dtype, long long np, double3 obs, double rmin, double rmax, int nbins,
                       const double* nbar, double P0, float* w, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  const double inv_dr = nbins / (rmax - rmin);
  const int blocks = (int)((np + 255) / 256 < 152 * 16 ? (np + 255) / 256 : 152 * 16);
  if (dtype == 0)
    fkp_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, np, obs, rmin, inv_dr, nbins, nbar, P0, w);
  else
    fkp_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, np, obs, rmin, inv_dr, nbins, nbar, P0, w);
  return cudaGetLastError();
}

cudaError_t launch_ratio(const float* num, const float* den, size_t n, double lo, double hi, double* partials,
                         int blocks, cudaStream_t st) {
  ratio_kernel<<<blocks, 256, 0, st>>>(num, den, n, lo, hi, partials);
  return cudaGetLastError();
}

}  // namespace rg

// ------------------------------------------------------------------------------------------------
// CIC deposit that allocates nothing (recon_cic_deposit_noalloc).  The only scratch it needs, the
// per-block partial sums of the weights, lives in a fixed file-scope device array; every device
// that loads the library holds these 32 KB until the process exits.
// ------------------------------------------------------------------------------------------------
namespace rg {
namespace {

constexpr int kNoAllocMaxBlocks = 4096;                    // partial sums in the static scratch
constexpr long long kNoAllocPerThread = 64;                // particles per thread at most
constexpr long long kNoAllocMaxParticles = (long long)kNoAllocMaxBlocks * 256 * kNoAllocPerThread;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per device.  The
// host-side name of a __device__ array is only a stand-in: kernels must be given this address.
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rg

extern "C" recon_status recon_cic_deposit_noalloc(const void* pos, int dtype, const float* w, int64_t n,
                                                  int nmesh, double box, float* rho, double* sum_w,
                                                  void* stream) {
  using namespace rg;
  if (n < 0 || (n > 0 && !pos) || !rho || !sum_w || nmesh < 2 || nmesh > 2048 || !(box > 0))
    return RECON_ERR_INVALID_ARG;
  if (dtype != RECON_F64 && dtype != RECON_F32) return RECON_ERR_INVALID_ARG;
  if (n > kNoAllocMaxParticles) return RECON_ERR_INVALID_ARG;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return RECON_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cells = (size_t)nmesh * nmesh * nmesh;
  if (cudaMemsetAsync(rho, 0, cells * sizeof(float), st) != cudaSuccess) return RECON_ERR_CUDA;
  if (n == 0) return cudaMemsetAsync(sum_w, 0, sizeof(double), st) == cudaSuccess ? RECON_OK : RECON_ERR_CUDA;
  long long blocks = (n + 255) / 256;
  if (blocks > kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
  if (launch_deposit(pos, dtype == RECON_F64 ? 0 : 1, w, n, nmesh, box, rho, scratch, (int)blocks, st) != cudaSuccess)
    return RECON_ERR_CUDA;
  if (launch_finalize(scratch, (int)blocks, 1, sum_w, 0, 0, st) != cudaSuccess) return RECON_ERR_CUDA;
  return RECON_OK;
}
