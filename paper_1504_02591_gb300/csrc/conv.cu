// conv.cu: Gaussian smoothing of the densities along x and y as periodic 1-D convolutions.
//
// The smoothing kernel of Sec. 3.1, S(k) = exp(-k^2 R^2 / 2), is a product of one factor per axis,
// so on the periodic mesh it is exactly three 1-D periodic convolutions with the real kernel
// g[t] = (1/N) sum_m exp(-k_m^2 R^2 / 2) exp(2 pi i m t / N) (computed on the host in float64).
// Applying it in configuration space keeps the float32 rounding relative to the local density:
// near the survey edge, where the smoothed random density falls to the mask threshold, a
// Fourier-space product would carry rounding of the order of the field's global magnitude.
// The z factor is applied inside the delta-forming Z pass; this file holds the x and y passes.
#include "conv.h"

namespace rg {

// One tile: every line of the axis (length n) for C adjacent z columns of one y (X pass) or one x
// (Y pass).  Lines are staged in shared memory; each output is written straight back to global
// memory (in place: all reads come from the staged copy).
template <int C>
__global__ void __launch_bounds__(256) conv_kernel(const ConvArgs a) {
  extern __shared__ float csm[];
  const int n = a.n;
  const int ntap = a.ntap;
  float* taps = csm;                         // ntap values
  float* s = csm + ((ntap + 3) & ~3);        // nf * n * C
  for (int j = threadIdx.x; j < ntap; j += blockDim.x) taps[j] = a.taps[j];

  const int zb = n / C;
  const int t = blockIdx.x;
  const int other = t / zb;                  // y (X pass) or x (Y pass)
  const int z0 = (t % zb) * C;
  const size_t nn = (size_t)n;
  size_t base, ls;
  if (a.axis == 0) {  // lines along x: (x N + y) N + z
    base = (size_t)other * nn + z0;
    ls = nn * nn;
  } else {            // lines along y
    base = (size_t)other * nn * nn + z0;
    ls = nn;
  }
  float cnt = 0.f;
  for (int q = 0; q < a.nf; ++q) {
    const float* src = a.f[q];
    for (int e = threadIdx.x; e < n * (C / 4); e += blockDim.x) {
      const int i = e / (C / 4), c4 = e % (C / 4);
      const float4 v = *reinterpret_cast<const float4*>(src + base + (size_t)i * ls + 4 * c4);
      if (a.count && q == a.nf - 1) cnt += (v.x > 0.f) + (v.y > 0.f) + (v.z > 0.f) + (v.w > 0.f);
      *reinterpret_cast<float4*>(s + (size_t)(q * n + i) * C + 4 * c4) = v;
    }
  }
  __syncthreads();
  for (int q = 0; q < a.nf; ++q) {
    const float* sq = s + (size_t)q * n * C;
    float* dst = a.f[q];
    for (int e = threadIdx.x; e < n * C; e += blockDim.x) {
      const int i = e / C, c = e % C;
      int idx = i + a.t0;
      if (idx < 0) idx += n;
      float acc = 0.f;
      for (int j = 0; j < ntap; ++j) {
        acc = fmaf(taps[j], sq[idx * C + c], acc);
        if (++idx == n) idx = 0;
      }
      dst[base + (size_t)i * ls + c] = acc;
    }
  }
  if (a.count) {
    __shared__ double sh[8];
    double v = cnt;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
      a.partials[2 * blockIdx.x + 0] = 0.0;
      a.partials[2 * blockIdx.x + 1] = r;
    }
  }
}

// Register-blocked form for kernels of at most KT taps, one field per CTA (blockIdx.y): the line is
// staged with its periodic continuation (s[p] = x[(p + t0) mod n], p < n + KT + V), the taps sit in
// registers (zero past ntap), and each thread slides over V consecutive outputs of one column, so
// every staged value is read once per V outputs instead of once per output.
template <int C, int KT, int V>
__global__ void __launch_bounds__(256) conv_blocked_kernel(const ConvArgs a) {
  extern __shared__ float csm[];
  constexpr int T = 256;
  const int n = a.n;
  const int len = n + KT + V;                // staged entries per line
  float tp[KT];
#pragma unroll
  for (int j = 0; j < KT; ++j) tp[j] = j < a.ntap ? a.taps[j] : 0.f;
  const int zb = n / C;
  const int t = blockIdx.x;
  const int other = t / zb;
  const int z0 = (t % zb) * C;
  const size_t nn = (size_t)n;
  size_t base, ls;
  if (a.axis == 0) {
    base = (size_t)other * nn + z0;
    ls = nn * nn;
  } else {
    base = (size_t)other * nn * nn + z0;
    ls = nn;
  }
  const int q = blockIdx.y;
  const bool count = a.count && q == a.nf - 1;
  float cnt = 0.f;
  {
    const float* src = a.f[q];
    for (int e = threadIdx.x; e < len * (C / 4); e += T) {
      const int p = e / (C / 4), c4 = e % (C / 4);
      int i = (p + a.t0) % n;
      if (i < 0) i += n;
      const float4 v = *reinterpret_cast<const float4*>(src + base + (size_t)i * ls + 4 * c4);
      if (count && p < n) cnt += (v.x > 0.f) + (v.y > 0.f) + (v.z > 0.f) + (v.w > 0.f);
      *reinterpret_cast<float4*>(csm + (size_t)p * C + 4 * c4) = v;
    }
  }
  __syncthreads();
  const int c = threadIdx.x % C;
  {
    float* dst = a.f[q];
    for (int i0 = (threadIdx.x / C) * V; i0 < n; i0 += (T / C) * V) {
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
#pragma unroll
      for (int j = 0; j < KT + V - 1; ++j) {
        const float x = csm[(size_t)(i0 + j) * C + c];
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (j - v >= 0 && j - v < KT) acc[v] = fmaf(tp[j - v], x, acc[v]);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) dst[base + (size_t)(i0 + v) * ls + c] = acc[v];
    }
  }
  if (count) {
    __shared__ double sh[8];
    double v = cnt;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
      a.partials[2 * blockIdx.x + 0] = 0.0;
      a.partials[2 * blockIdx.x + 1] = r;
    }
  }
}

constexpr int kConvV = 8;

// Adjacent z columns per tile: 128-byte rows where the staged line of a field still leaves room for
// three CTAs per SM.
int conv_cols(int n) { return n >= 1024 ? 8 : (n >= 256 ? 32 : 16); }

int conv_blocks(int n) { return n * (n / conv_cols(n)); }

static int conv_kt(int n, int ntap) {
  if (n % (256 / conv_cols(n) * kConvV) != 0) return 0;   // every thread's blocks of V outputs fit the line
  return ntap <= 32 ? 32 : (ntap <= 64 ? 64 : 0);
}

size_t conv_smem(int n, int nf, int ntap) {
  const int kt = conv_kt(n, ntap);
  if (kt) return sizeof(float) * (size_t)(n + kt + kConvV) * conv_cols(n);   // one field per CTA
  return sizeof(float) * (((size_t)ntap + 3) / 4 * 4 + (size_t)nf * n * conv_cols(n));
}

// The y pass reads 2 KB-strided lines, where 64-byte row segments still stream well: 16 columns
// (half the staged line, twice the CTAs per SM) cut the x and y passes together from 1.52 to 1.44 ms
// at 512^3.
constexpr int kConvYCols = 16;

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t st) {
  const int C = (a.axis == 1 && a.n >= 256 && a.n < 1024 && a.n % (256 / kConvYCols * kConvV) == 0)
                    ? kConvYCols : conv_cols(a.n);
  const int kt = conv_kt(a.n, a.ntap);
  const size_t smem = kt ? sizeof(float) * (size_t)(a.n + kt + kConvV) * C
                         : sizeof(float) * (((size_t)a.ntap + 3) / 4 * 4 + (size_t)a.nf * a.n * C);
  const void* k;
  if (kt == 32)
    k = (C == 32) ? (const void*)conv_blocked_kernel<32, 32, kConvV>
                  : (C == 16) ? (const void*)conv_blocked_kernel<16, 32, kConvV> : (const void*)conv_blocked_kernel<8, 32, kConvV>;
  else if (kt == 64)
    k = (C == 32) ? (const void*)conv_blocked_kernel<32, 64, kConvV>
                  : (C == 16) ? (const void*)conv_blocked_kernel<16, 64, kConvV> : (const void*)conv_blocked_kernel<8, 64, kConvV>;
  else
    k = (C == 32) ? (const void*)conv_kernel<32> : (C == 16) ? (const void*)conv_kernel<16> : (const void*)conv_kernel<8>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<ConvArgs*>(&a)};
  return cudaLaunchKernel(k, dim3(a.n * (a.n / C), kt ? a.nf : 1), dim3(256), args, smem, st);
}

}  // namespace rg
