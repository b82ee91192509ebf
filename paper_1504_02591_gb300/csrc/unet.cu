// unet.cu: the learned warm start — a small periodic 3-D U-Net with its own forward, backward and
// AdamW kernels (float32 accumulation; activations stored as bfloat16 or float32).
//
// Network (3 levels, widths c1/2c1/4c1): two 3x3x3 conv+ReLU per level, 2x2x2 average pooling down,
// nearest-neighbour 2x upsampling up, skip connections by channel concatenation, and a 1x1x1 head
// whose output is added to the last input channel (the radial displacement of the Eq. approx2
// start), so the network predicts the correction that brings the start to the converged solution
// of Eq. Nusser.  Tensors are channels-last [voxel][channel] on a periodic n^3 grid; a 3x3x3 kernel
// w[tap][cin][cout] computes y[v][co] = b[co] + sum_tap sum_ci x[v + d(tap)][ci] w[tap][ci][co].
#include <cuda_bf16.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/recon.h"
#include "unet_tc.h"

namespace rg {
namespace {

typedef __nv_bfloat16 bf16;

template <typename T>
__device__ __forceinline__ float tof(T v);
template <>
__device__ __forceinline__ float tof<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tof<bf16>(bf16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T fromf(float v);
template <>
__device__ __forceinline__ float fromf<float>(float v) { return v; }
template <>
__device__ __forceinline__ bf16 fromf<bf16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void tap_offset(int t, int ntap, int& dx, int& dy, int& dz) {
  if (ntap == 27) {
    dx = t / 9 - 1;
    dy = (t / 3) % 3 - 1;
    dz = t % 3 - 1;
  } else {
    dx = dy = dz = 0;
  }
}

// ---- convolution forward: y = act(b + conv(concat(xa, xb))) (+ res for the head) ----------------
template <typename T, int COUT>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const T* __restrict__ xa, int ca, const T* __restrict__ xb,
                                                       int cb, const T* __restrict__ w, const float* __restrict__ bias,
                                                       int ntap, int n, int relu, const float* __restrict__ res,
                                                       int res_stride, T* __restrict__ y, float* __restrict__ yf) {
  extern __shared__ float wsm[];
  const int cin = ca + cb;
  const long long nv = (long long)n * n * n;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = bias[co];
  int ix = 0, iy = 0, iz = 0;
  if (v < nv) {
    ix = (int)(v / ((long long)n * n));
    iy = (int)((v / n) % n);
    iz = (int)(v % n);
  }
  for (int t = 0; t < ntap; ++t) {
    __syncthreads();
    for (int e = threadIdx.x; e < cin * COUT; e += blockDim.x) wsm[e] = tof(w[(size_t)t * cin * COUT + e]);
    __syncthreads();
    if (v < nv) {
      int dx, dy, dz;
      tap_offset(t, ntap, dx, dy, dz);
      const long long u = ((long long)wrapc(ix + dx, n) * n + wrapc(iy + dy, n)) * n + wrapc(iz + dz, n);
      const T* pa = xa + u * ca;
      for (int ci = 0; ci < ca; ++ci) {
        const float xv = tof(pa[ci]);
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(xv, wsm[ci * COUT + co], acc[co]);
      }
      if (cb) {
        const T* pb = xb + u * cb;
        for (int ci = 0; ci < cb; ++ci) {
          const float xv = tof(pb[ci]);
#pragma unroll
          for (int co = 0; co < COUT; ++co) acc[co] = fmaf(xv, wsm[(ca + ci) * COUT + co], acc[co]);
        }
      }
    }
  }
  if (v < nv) {
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      float o = acc[co];
      if (relu) o = fmaxf(o, 0.f);
      if (res) o += res[v * res_stride];
      if (y) y[v * COUT + co] = fromf<T>(o);
      if (yf) yf[v * COUT + co] = o;
    }
  }
}

// ---- gradient w.r.t. the input: gx[v][ci] = sum_t sum_co gy[v - d(t)][co] w[t][ci][co] ---------
constexpr int kDChunk = 16;
template <typename T>
__global__ void __launch_bounds__(128) conv_dgrad_kernel(const float* __restrict__ gy, int cout,
                                                         const T* __restrict__ w, int ca, int cb, int ntap, int n,
                                                         float* __restrict__ gxa, float* __restrict__ gxb, int accum_b) {
  extern __shared__ float wsm[];   // kDChunk x cout
  const int cin = ca + cb;
  const int c0 = blockIdx.y * kDChunk;
  const long long nv = (long long)n * n * n;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[kDChunk];
#pragma unroll
  for (int k = 0; k < kDChunk; ++k) acc[k] = 0.f;
  int ix = 0, iy = 0, iz = 0;
  if (v < nv) {
    ix = (int)(v / ((long long)n * n));
    iy = (int)((v / n) % n);
    iz = (int)(v % n);
  }
  for (int t = 0; t < ntap; ++t) {
    __syncthreads();
    for (int e = threadIdx.x; e < kDChunk * cout; e += blockDim.x) {
      const int cl = e / cout, co = e % cout;
      wsm[e] = (c0 + cl < cin) ? tof(w[((size_t)t * cin + c0 + cl) * cout + co]) : 0.f;
    }
    __syncthreads();
    if (v < nv) {
      int dx, dy, dz;
      tap_offset(t, ntap, dx, dy, dz);
      const long long u = ((long long)wrapc(ix - dx, n) * n + wrapc(iy - dy, n)) * n + wrapc(iz - dz, n);
      const float* g = gy + u * cout;
      for (int co = 0; co < cout; ++co) {
        const float gv = g[co];
#pragma unroll
        for (int k = 0; k < kDChunk; ++k) acc[k] = fmaf(gv, wsm[k * cout + co], acc[k]);
      }
    }
  }
  if (v < nv) {
#pragma unroll
    for (int k = 0; k < kDChunk; ++k) {
      const int ci = c0 + k;
      if (ci < ca) {
        gxa[v * ca + ci] = acc[k];
      } else if (ci < cin) {
        float* p = gxb + v * cb + (ci - ca);
        *p = accum_b ? *p + acc[k] : acc[k];
      }
    }
  }
}

// ---- gradient w.r.t. the weights: gw[t][ci][co] += sum_v x[v + d(t)][ci] gy[v][co] ---------------
constexpr int kWVox = 32;       // voxels staged per round
constexpr int kWPairs = 16;     // (ci, co) pairs per thread (cin * cout <= 4096)
template <typename T>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const T* __restrict__ xa, int ca, const T* __restrict__ xb,
                                                         int cb, const float* __restrict__ gy, int cout, int ntap, int n,
                                                         float* __restrict__ gw) {
  extern __shared__ float sm[];
  const int cin = ca + cb;
  float* xs = sm;                       // kWVox x cin
  float* gs = sm + kWVox * cin;         // kWVox x cout
  const int t = blockIdx.y;
  int dx, dy, dz;
  tap_offset(t, ntap, dx, dy, dz);
  const long long nv = (long long)n * n * n;
  const int P = cin * cout;
  float acc[kWPairs];
#pragma unroll
  for (int k = 0; k < kWPairs; ++k) acc[k] = 0.f;
  for (long long v0 = (long long)blockIdx.x * kWVox; v0 < nv; v0 += (long long)gridDim.x * kWVox) {
    __syncthreads();
    for (int e = threadIdx.x; e < kWVox * cin; e += blockDim.x) {
      const int lv = e / cin, ci = e % cin;
      const long long v = v0 + lv;
      float xv = 0.f;
      if (v < nv) {
        const int ix = (int)(v / ((long long)n * n)), iy = (int)((v / n) % n), iz = (int)(v % n);
        const long long u = ((long long)wrapc(ix + dx, n) * n + wrapc(iy + dy, n)) * n + wrapc(iz + dz, n);
        xv = ci < ca ? tof(xa[u * ca + ci]) : tof(xb[u * cb + (ci - ca)]);
      }
      xs[e] = xv;
    }
    for (int e = threadIdx.x; e < kWVox * cout; e += blockDim.x) {
      const long long v = v0 + e / cout;
      gs[e] = v < nv ? gy[v * cout + e % cout] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kWPairs; ++k) {
      const int p = threadIdx.x + k * 256;
      if (p < P) {
        const int ci = p / cout, co = p % cout;
        float a = acc[k];
        for (int lv = 0; lv < kWVox; ++lv) a = fmaf(xs[lv * cin + ci], gs[lv * cout + co], a);
        acc[k] = a;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kWPairs; ++k) {
    const int p = threadIdx.x + k * 256;
    if (p < P) atomicAdd(gw + (size_t)t * P + p, acc[k]);
  }
}

__global__ void bias_grad_kernel(const float* __restrict__ gy, int cout, long long nv, float* __restrict__ gb) {
  __shared__ float sh[256];
  for (int co = 0; co < cout; ++co) {
    float s = 0.f;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x)
      s += gy[v * cout + co];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(gb + co, sh[0]);
    __syncthreads();
  }
}

template <typename T>
__global__ void relu_backward_kernel(float* __restrict__ g, const T* __restrict__ y, long long m) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    if (!(tof(y[i]) > 0.f)) g[i] = 0.f;
}

// 2x2x2 average pooling: coarse n/2 grid
template <typename T>
__global__ void pool_kernel(const T* __restrict__ x, int c, int n, T* __restrict__ y) {
  const int m = n / 2;
  const long long tot = (long long)m * m * m * c;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const long long cv = i / c;
    const int X = (int)(cv / ((long long)m * m)), Y = (int)((cv / m) % m), Z = (int)(cv % m);
    float s = 0.f;
    for (int a = 0; a < 8; ++a) {
      const long long f = ((long long)(2 * X + (a >> 2)) * n + (2 * Y + ((a >> 1) & 1))) * n + (2 * Z + (a & 1));
      s += tof(x[f * c + ch]);
    }
    y[i] = fromf<T>(0.125f * s);
  }
}

__global__ void pool_backward_kernel(const float* __restrict__ g, int c, int n, float* __restrict__ gx, int accum) {
  const long long tot = (long long)n * n * n * c;
  const int m = n / 2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const long long f = i / c;
    const int x = (int)(f / ((long long)n * n)), y = (int)((f / n) % n), z = (int)(f % n);
    const float v = 0.125f * g[(((long long)(x >> 1) * m + (y >> 1)) * m + (z >> 1)) * c + ch];
    gx[i] = accum ? gx[i] + v : v;
  }
}

// nearest-neighbour 2x upsampling from the coarse n/2 grid to n
template <typename T>
__global__ void up_kernel(const T* __restrict__ x, int c, int n, T* __restrict__ y) {
  const long long tot = (long long)n * n * n * c;
  const int m = n / 2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const long long f = i / c;
    const int X = (int)(f / ((long long)n * n)), Y = (int)((f / n) % n), Z = (int)(f % n);
    y[i] = x[(((long long)(X >> 1) * m + (Y >> 1)) * m + (Z >> 1)) * c + ch];
  }
}

__global__ void up_backward_kernel(const float* __restrict__ g, int c, int n, float* __restrict__ gx) {
  const int m = n / 2;
  const long long tot = (long long)m * m * m * c;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    const long long cv = i / c;
    const int X = (int)(cv / ((long long)m * m)), Y = (int)((cv / m) % m), Z = (int)(cv % m);
    float s = 0.f;
    for (int a = 0; a < 8; ++a) {
      const long long f = ((long long)(2 * X + (a >> 2)) * n + (2 * Y + ((a >> 1) & 1))) * n + (2 * Z + (a & 1));
      s += g[f * c + ch];
    }
    gx[i] = s;
  }
}

template <typename T>
__global__ void to_t_kernel(const float* __restrict__ x, T* __restrict__ y, long long m) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    y[i] = fromf<T>(x[i]);
}

// network input for the tensor-core path: 5 float32 channels -> 8 bf16 channels (16 bytes a voxel)
__global__ void to_x8_kernel(const float* __restrict__ x, int cin, long long nv, bf16* __restrict__ y) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 o[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16_rn(c < cin ? x[v * cin + c] : 0.f);
    *reinterpret_cast<uint4*>(y + v * 8) = *reinterpret_cast<const uint4*>(o);
  }
}

// mean squared error: g = 2 (y - t) / m, loss = sum (y - t)^2 / m (float64 accumulation)
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long m, float* __restrict__ g,
                           double* __restrict__ loss) {
  __shared__ double sh[256];
  double s = 0.0;
  const float sc = 2.f / (float)m;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = sc * d;
    s += (double)d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, sh[0] / (double)m);
}

// decoupled weight decay Adam on the float32 master weights; refreshes the stored-type copy
template <typename T>
__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                             float* __restrict__ m2, const unsigned char* __restrict__ decay, T* __restrict__ pt,
                             long long np, float lr, float wd, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float w = p[i] - lr * ((a / c1) / (sqrtf(b / c2) + 1e-8f) + (decay[i] ? wd * p[i] : 0.f));
    p[i] = w;
    pt[i] = fromf<T>(w);
  }
}

int grid_for(long long m, int threads = 256) {
  long long b = (m + threads - 1) / threads;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

struct Spec {
  const char* name;
  int cin, cout, ntap;
};

}  // namespace
}  // namespace rg

using namespace rg;

struct recon_unet {
  int c1 = 16, cin = 5, bf16 = 1, n_alloc = 0, step = 0;
  cudaStream_t st = nullptr;
  std::vector<Spec> spec;
  std::vector<size_t> woff, boff;
  size_t np = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  unsigned char* decay = nullptr;
  void* pt = nullptr;                  // stored-type copy of the parameters
  void* acts = nullptr;                // activations (stored type) for n_alloc
  float* grads = nullptr;              // activation gradients for n_alloc
  float* y = nullptr;                  // network output (float)
  double* loss = nullptr;
  std::string err;
  // tensor-core forward
  int use_tc = 1;
  int* dev_err = nullptr;              // set by a tensor-core kernel whose wait timed out
  void* wpack = nullptr;               // packed weight tiles of the layers on the tensor-core path
  size_t wpack_cap = 0;
  rg::tc::ConvPlan plan[10];
  bool plan_ok[10] = {};
  size_t pack_off[10] = {};
  int plan_n = 0;
  unsigned pver = 1, packed_ver = 0;   // parameter version, version the packed tiles were made from
  int last_n = 0;                      // side of the last forward
  long long launches = 0;              // kernels launched by recon_unet_forward (all calls)
  bool head_fused = false;             // last forward fused the head into layer 9 (d1b not stored)
};

namespace {

void make_spec(recon_unet* u) {
  const int c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1, ci = u->cin;
  u->spec = {{"enc1a", ci, c1, 27}, {"enc1b", c1, c1, 27}, {"enc2a", c1, c2, 27}, {"enc2b", c2, c2, 27},
             {"bota", c2, c3, 27},  {"botb", c3, c3, 27},  {"dec2a", c3 + c2, c2, 27}, {"dec2b", c2, c2, 27},
             {"dec1a", c2 + c1, c1, 27}, {"dec1b", c1, c1, 27}, {"head", c1, 1, 1}};
  u->woff.clear();
  u->boff.clear();
  size_t o = 0;
  for (auto& s : u->spec) {
    u->woff.push_back(o);
    o += (size_t)s.ntap * s.cin * s.cout;
    u->boff.push_back(o);
    o += s.cout;
  }
  u->np = o;
}

// activation layout for one grid of side n (offsets in elements of the stored type)
struct Acts {
  size_t x, a1a, a1b, p1, a2a, a2b, p2, a3a, a3b, u3, d2a, d2b, u2, d1a, d1b, x8, total;
};
Acts act_layout(const recon_unet* u, int n) {
  const size_t V1 = (size_t)n * n * n, V2 = V1 / 8, V3 = V1 / 64;
  const size_t c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1;
  Acts a{};
  size_t o = 0;
  auto take = [&](size_t k) { size_t r = o; o += (k + 127) & ~(size_t)127; return r; };
  a.x = take(V1 * u->cin);
  a.a1a = take(V1 * c1); a.a1b = take(V1 * c1); a.p1 = take(V2 * c1);
  a.a2a = take(V2 * c2); a.a2b = take(V2 * c2); a.p2 = take(V3 * c2);
  a.a3a = take(V3 * c3); a.a3b = take(V3 * c3); a.u3 = take(V2 * c3);
  a.d2a = take(V2 * c2); a.d2b = take(V2 * c2); a.u2 = take(V1 * c2);
  a.d1a = take(V1 * c1); a.d1b = take(V1 * c1);
  a.x8 = take(V1 * 8);
  a.total = o;
  return a;
}
struct Grads {
  size_t gy, gd1b, gd1a, gu2, gs1, gd2b, gd2a, gu3, gs2, ga3b, ga3a, gp2, ga2a, gp1, ga1a, total;
};
Grads grad_layout(const recon_unet* u, int n) {
  const size_t V1 = (size_t)n * n * n, V2 = V1 / 8, V3 = V1 / 64;
  const size_t c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1;
  Grads g{};
  size_t o = 0;
  auto take = [&](size_t k) { size_t r = o; o += (k + 63) & ~(size_t)63; return r; };
  g.gy = take(V1); g.gd1b = take(V1 * c1); g.gd1a = take(V1 * c1); g.gu2 = take(V1 * c2); g.gs1 = take(V1 * c1);
  g.gd2b = take(V2 * c2); g.gd2a = take(V2 * c2); g.gu3 = take(V2 * c3); g.gs2 = take(V2 * c2);
  g.ga3b = take(V3 * c3); g.ga3a = take(V3 * c3); g.gp2 = take(V3 * c2); g.ga2a = take(V2 * c2);
  g.gp1 = take(V2 * c1); g.ga1a = take(V1 * c1);
  g.total = o;
  return g;
}

#define UN_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      u->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
      return RECON_ERR_CUDA;                                            \
    }                                                                   \
  } while (0)

recon_status ensure(recon_unet* u, int n, bool train) {
  if (n < 8 || n % 8 != 0) return RECON_ERR_INVALID_ARG;
  if (n <= u->n_alloc && (!train || u->grads)) return RECON_OK;
  const int nn = n > u->n_alloc ? n : u->n_alloc;
  if (u->acts) cudaFree(u->acts);
  if (u->grads) cudaFree(u->grads);
  if (u->y) cudaFree(u->y);
  u->acts = nullptr;
  u->grads = nullptr;
  u->y = nullptr;
  const size_t es = u->bf16 ? 2 : 4;
  if (cudaMalloc(&u->acts, act_layout(u, nn).total * es) != cudaSuccess ||
      cudaMalloc(&u->y, (size_t)nn * nn * nn * sizeof(float)) != cudaSuccess ||
      (train && cudaMalloc(&u->grads, grad_layout(u, nn).total * sizeof(float)) != cudaSuccess)) {
    cudaGetLastError();
    return RECON_ERR_OOM;
  }
  u->n_alloc = nn;
  return RECON_OK;
}

template <typename T>
cudaError_t conv_fwd(recon_unet* u, int li, const T* xa, int ca, const T* xb, int cb, int n, int relu,
                     const float* res, int res_stride, T* y, float* yf) {
  const Spec& s = u->spec[li];
  const T* w = static_cast<const T*>(u->pt) + u->woff[li];
  const float* b = u->p + u->boff[li];
  const long long nv = (long long)n * n * n;
  const int blocks = (int)((nv + 127) / 128);
  const size_t smem = sizeof(float) * s.cin * s.cout;
  switch (s.cout) {
#define UN_CASE(C)                                                                                   \
  case C:                                                                                           \
    conv_fwd_kernel<T, C><<<blocks, 128, smem, u->st>>>(xa, ca, xb, cb, w, b, s.ntap, n, relu, res, res_stride, y, yf); \
    break;
    UN_CASE(1) UN_CASE(8) UN_CASE(16) UN_CASE(32) UN_CASE(64) UN_CASE(128)
#undef UN_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t conv_back(recon_unet* u, int li, const T* xa, int ca, const T* xb, int cb, const float* gy, int n,
                      float* gxa, float* gxb, int accum_b) {
  const Spec& s = u->spec[li];
  const T* w = static_cast<const T*>(u->pt) + u->woff[li];
  const long long nv = (long long)n * n * n;
  float* gw = u->g + u->woff[li];
  float* gb = u->g + u->boff[li];
  if (s.cin * s.cout > 256 * kWPairs) return cudaErrorInvalidValue;
  const int wblocks = (int)((nv + kWVox - 1) / kWVox < 304 ? (nv + kWVox - 1) / kWVox : 304);
  conv_wgrad_kernel<T><<<dim3(wblocks, s.ntap), 256, sizeof(float) * kWVox * (s.cin + s.cout), u->st>>>(
      xa, ca, xb, cb, gy, s.cout, s.ntap, n, gw);
  bias_grad_kernel<<<grid_for(nv) < 304 ? grid_for(nv) : 304, 256, 0, u->st>>>(gy, s.cout, nv, gb);
  if (gxa || gxb) {
    dim3 grid((unsigned)((nv + 127) / 128), (unsigned)((s.cin + kDChunk - 1) / kDChunk));
    conv_dgrad_kernel<T><<<grid, 128, sizeof(float) * kDChunk * s.cout, u->st>>>(gy, s.cout, w, ca, cb, s.ntap, n,
                                                                                 gxa, gxb, accum_b);
  }
  return cudaGetLastError();
}

template <typename T>
recon_status forward_t(recon_unet* u, const float* x, int n, float* out) {
  const Acts A = act_layout(u, n);
  T* a = static_cast<T*>(u->acts);
  const int c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1, n2 = n / 2, n4 = n / 4;
  const long long V1 = (long long)n * n * n;
  to_t_kernel<T><<<grid_for(V1 * u->cin), 256, 0, u->st>>>(x, a + A.x, V1 * u->cin);
  UN_CUDA(conv_fwd<T>(u, 0, a + A.x, u->cin, nullptr, 0, n, 1, nullptr, 0, a + A.a1a, nullptr));
  UN_CUDA(conv_fwd<T>(u, 1, a + A.a1a, c1, nullptr, 0, n, 1, nullptr, 0, a + A.a1b, nullptr));
  pool_kernel<T><<<grid_for(V1 / 8 * c1), 256, 0, u->st>>>(a + A.a1b, c1, n, a + A.p1);
  UN_CUDA(conv_fwd<T>(u, 2, a + A.p1, c1, nullptr, 0, n2, 1, nullptr, 0, a + A.a2a, nullptr));
  UN_CUDA(conv_fwd<T>(u, 3, a + A.a2a, c2, nullptr, 0, n2, 1, nullptr, 0, a + A.a2b, nullptr));
  pool_kernel<T><<<grid_for(V1 / 64 * c2), 256, 0, u->st>>>(a + A.a2b, c2, n2, a + A.p2);
  UN_CUDA(conv_fwd<T>(u, 4, a + A.p2, c2, nullptr, 0, n4, 1, nullptr, 0, a + A.a3a, nullptr));
  UN_CUDA(conv_fwd<T>(u, 5, a + A.a3a, c3, nullptr, 0, n4, 1, nullptr, 0, a + A.a3b, nullptr));
  up_kernel<T><<<grid_for(V1 / 8 * c3), 256, 0, u->st>>>(a + A.a3b, c3, n2, a + A.u3);
  UN_CUDA(conv_fwd<T>(u, 6, a + A.u3, c3, a + A.a2b, c2, n2, 1, nullptr, 0, a + A.d2a, nullptr));
  UN_CUDA(conv_fwd<T>(u, 7, a + A.d2a, c2, nullptr, 0, n2, 1, nullptr, 0, a + A.d2b, nullptr));
  up_kernel<T><<<grid_for(V1 * c2), 256, 0, u->st>>>(a + A.d2b, c2, n, a + A.u2);
  UN_CUDA(conv_fwd<T>(u, 8, a + A.u2, c2, a + A.a1b, c1, n, 1, nullptr, 0, a + A.d1a, nullptr));
  UN_CUDA(conv_fwd<T>(u, 9, a + A.d1a, c1, nullptr, 0, n, 1, nullptr, 0, a + A.d1b, nullptr));
  UN_CUDA(conv_fwd<T>(u, 10, a + A.d1b, c1, nullptr, 0, n, 0, x + (u->cin - 1), u->cin, nullptr, out));
  return RECON_OK;
}

// Tensor-core plans for the ten 3x3x3 layers at grid side n (levels n, n/2, n/4), and the packed
// weight tiles; a layer whose level does not fit the tensor-core tiling stays on the CUDA cores.
recon_status tc_prepare(recon_unet* u, int n) {
  const int c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1, n2 = n / 2, n4 = n / 4;
  if (u->plan_n != n) {
    struct L {
      int n, c0, up0, c1, cin, cout;
    };
    const L ls[10] = {{n, 8, 0, 0, u->cin, c1},      {n, c1, 0, 0, c1, c1},         {n2, c1, 0, 0, c1, c2},
                      {n2, c2, 0, 0, c2, c2},        {n4, c2, 0, 0, c2, c3},        {n4, c3, 0, 0, c3, c3},
                      {n2, c3, 1, c2, c3 + c2, c2},  {n2, c2, 0, 0, c2, c2},        {n, c2, 1, c1, c2 + c1, c1},
                      {n, c1, 0, 0, c1, c1}};
    size_t off = 0;
    for (int l = 0; l < 10; ++l) {
      u->plan_ok[l] = tc::plan_conv(ls[l].n, ls[l].c0, ls[l].up0, ls[l].c1, ls[l].cin, ls[l].cout, &u->plan[l]);
      u->pack_off[l] = off;
      if (u->plan_ok[l]) off += (u->plan[l].packed_elems + 127) / 128 * 128;
    }
    if (off * sizeof(bf16) > u->wpack_cap) {
      cudaFree(u->wpack);
      u->wpack = nullptr;
      u->wpack_cap = 0;
      if (cudaMalloc(&u->wpack, off * sizeof(bf16)) != cudaSuccess) {
        cudaGetLastError();
        u->plan_n = 0;
        return RECON_ERR_OOM;
      }
      u->wpack_cap = off * sizeof(bf16);
    }
    u->plan_n = n;
    u->packed_ver = 0;
  }
  if (u->packed_ver != u->pver) {
    const bf16* w = static_cast<const bf16*>(u->pt);
    for (int l = 0; l < 10; ++l)
      if (u->plan_ok[l]) {
        ++u->launches;
        UN_CUDA(tc::pack_weights(u->plan[l], w + u->woff[l], static_cast<bf16*>(u->wpack) + u->pack_off[l], u->st));
      }
    u->packed_ver = u->pver;
  }
  return RECON_OK;
}

// Inference forward with bf16 storage: the same network and rounding points as forward_t<bf16>,
// with the convolutions on the tensor cores where the level allows, the upsampling folded into the
// loads of the decoder convolutions and the 1x1 head folded into the last convolution.
recon_status forward_tc(recon_unet* u, const float* x, int n, float* out) {
  recon_status rs = tc_prepare(u, n);
  if (rs != RECON_OK) return rs;
  const Acts A = act_layout(u, n);
  bf16* a = static_cast<bf16*>(u->acts);
  const bf16* wp = static_cast<const bf16*>(u->wpack);
  const int c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1, n2 = n / 2, n4 = n / 4;
  const long long V1 = (long long)n * n * n;
  auto run = [&](int l, const bf16* s0, const bf16* s1, bf16* y) -> cudaError_t {
    ++u->launches;
    tc::ConvIO io;
    io.src0 = s0;
    io.src1 = s1;
    io.wpack = wp + u->pack_off[l];
    io.bias = u->p + u->boff[l];
    io.out = y;
    io.err = u->dev_err;
    return tc::conv_forward(u->plan[l], io, u->st);
  };
  auto plain = [&](int l, const bf16* s0, int ca, bf16* y, int nl) -> cudaError_t {
    if (u->plan_ok[l]) return run(l, s0, nullptr, y);
    ++u->launches;
    return conv_fwd<bf16>(u, l, s0, ca, nullptr, 0, nl, 1, nullptr, 0, y, nullptr);
  };
  u->launches += 3;   // input conversion and the two poolings
  if (u->plan_ok[0]) {
    to_x8_kernel<<<grid_for(V1), 256, 0, u->st>>>(x, u->cin, V1, a + A.x8);
    UN_CUDA(run(0, a + A.x8, nullptr, a + A.a1a));
  } else {
    to_t_kernel<bf16><<<grid_for(V1 * u->cin), 256, 0, u->st>>>(x, a + A.x, V1 * u->cin);
    UN_CUDA(conv_fwd<bf16>(u, 0, a + A.x, u->cin, nullptr, 0, n, 1, nullptr, 0, a + A.a1a, nullptr));
  }
  UN_CUDA(plain(1, a + A.a1a, c1, a + A.a1b, n));
  pool_kernel<bf16><<<grid_for(V1 / 8 * c1), 256, 0, u->st>>>(a + A.a1b, c1, n, a + A.p1);
  UN_CUDA(plain(2, a + A.p1, c1, a + A.a2a, n2));
  UN_CUDA(plain(3, a + A.a2a, c2, a + A.a2b, n2));
  pool_kernel<bf16><<<grid_for(V1 / 64 * c2), 256, 0, u->st>>>(a + A.a2b, c2, n2, a + A.p2);
  UN_CUDA(plain(4, a + A.p2, c2, a + A.a3a, n4));
  UN_CUDA(plain(5, a + A.a3a, c3, a + A.a3b, n4));
  if (u->plan_ok[6]) {
    UN_CUDA(run(6, a + A.a3b, a + A.a2b, a + A.d2a));
  } else {
    u->launches += 2;
    up_kernel<bf16><<<grid_for(V1 / 8 * c3), 256, 0, u->st>>>(a + A.a3b, c3, n2, a + A.u3);
    UN_CUDA(conv_fwd<bf16>(u, 6, a + A.u3, c3, a + A.a2b, c2, n2, 1, nullptr, 0, a + A.d2a, nullptr));
  }
  UN_CUDA(plain(7, a + A.d2a, c2, a + A.d2b, n2));
  if (u->plan_ok[8]) {
    UN_CUDA(run(8, a + A.d2b, a + A.a1b, a + A.d1a));
  } else {
    u->launches += 2;
    up_kernel<bf16><<<grid_for(V1 * c2), 256, 0, u->st>>>(a + A.d2b, c2, n, a + A.u2);
    UN_CUDA(conv_fwd<bf16>(u, 8, a + A.u2, c2, a + A.a1b, c1, n, 1, nullptr, 0, a + A.d1a, nullptr));
  }
  u->head_fused = u->plan_ok[9] && u->plan[9].orient == 0;
  if (u->head_fused) {
    tc::ConvIO io;
    io.src0 = a + A.d1a;
    io.wpack = wp + u->pack_off[9];
    io.bias = u->p + u->boff[9];
    io.head_w = static_cast<const bf16*>(u->pt) + u->woff[10];
    io.head_b = u->p + u->boff[10];
    io.res = x + (u->cin - 1);
    io.res_stride = u->cin;
    io.yout = out;
    io.err = u->dev_err;
    ++u->launches;
    UN_CUDA(tc::conv_forward(u->plan[9], io, u->st));
  } else {
    ++u->launches;
    UN_CUDA(plain(9, a + A.d1a, c1, a + A.d1b, n));
    UN_CUDA(conv_fwd<bf16>(u, 10, a + A.d1b, c1, nullptr, 0, n, 0, x + (u->cin - 1), u->cin, nullptr, out));
  }
  int flag = 0;
  UN_CUDA(cudaMemcpyAsync(&flag, u->dev_err, sizeof(int), cudaMemcpyDeviceToHost, u->st));
  UN_CUDA(cudaStreamSynchronize(u->st));
  if (flag) {
    cudaMemsetAsync(u->dev_err, 0, sizeof(int), u->st);
    u->err = "tensor-core convolution: a pipeline wait timed out";
    return RECON_ERR_CUDA;
  }
  return RECON_OK;
}

template <typename T>
recon_status backward_t(recon_unet* u, const float* x, const float* target, int n, double* loss) {
  recon_status rs = forward_t<T>(u, x, n, u->y);
  if (rs != RECON_OK) return rs;
  const Acts A = act_layout(u, n);
  const Grads G = grad_layout(u, n);
  const T* a = static_cast<const T*>(u->acts);
  float* g = u->grads;
  const int c1 = u->c1, c2 = 2 * c1, c3 = 4 * c1, n2 = n / 2, n4 = n / 4;
  const long long V1 = (long long)n * n * n, V2 = V1 / 8, V3 = V1 / 64;
  UN_CUDA(cudaMemsetAsync(u->g, 0, u->np * sizeof(float), u->st));
  UN_CUDA(cudaMemsetAsync(u->loss, 0, sizeof(double), u->st));
  mse_kernel<<<grid_for(V1) < 304 ? grid_for(V1) : 304, 256, 0, u->st>>>(u->y, target, V1, g + G.gy, u->loss);
  auto relu_b = [&](float* gp, const T* yp, long long m) {
    relu_backward_kernel<T><<<grid_for(m), 256, 0, u->st>>>(gp, yp, m);
  };
  UN_CUDA(conv_back<T>(u, 10, a + A.d1b, c1, nullptr, 0, g + G.gy, n, g + G.gd1b, nullptr, 0));
  relu_b(g + G.gd1b, a + A.d1b, V1 * c1);
  UN_CUDA(conv_back<T>(u, 9, a + A.d1a, c1, nullptr, 0, g + G.gd1b, n, g + G.gd1a, nullptr, 0));
  relu_b(g + G.gd1a, a + A.d1a, V1 * c1);
  UN_CUDA(conv_back<T>(u, 8, a + A.u2, c2, a + A.a1b, c1, g + G.gd1a, n, g + G.gu2, g + G.gs1, 0));
  up_backward_kernel<<<grid_for(V2 * c2), 256, 0, u->st>>>(g + G.gu2, c2, n, g + G.gd2b);
  relu_b(g + G.gd2b, a + A.d2b, V2 * c2);
  UN_CUDA(conv_back<T>(u, 7, a + A.d2a, c2, nullptr, 0, g + G.gd2b, n2, g + G.gd2a, nullptr, 0));
  relu_b(g + G.gd2a, a + A.d2a, V2 * c2);
  UN_CUDA(conv_back<T>(u, 6, a + A.u3, c3, a + A.a2b, c2, g + G.gd2a, n2, g + G.gu3, g + G.gs2, 0));
  up_backward_kernel<<<grid_for(V3 * c3), 256, 0, u->st>>>(g + G.gu3, c3, n2, g + G.ga3b);
  relu_b(g + G.ga3b, a + A.a3b, V3 * c3);
  UN_CUDA(conv_back<T>(u, 5, a + A.a3a, c3, nullptr, 0, g + G.ga3b, n4, g + G.ga3a, nullptr, 0));
  relu_b(g + G.ga3a, a + A.a3a, V3 * c3);
  UN_CUDA(conv_back<T>(u, 4, a + A.p2, c2, nullptr, 0, g + G.ga3a, n4, g + G.gp2, nullptr, 0));
  pool_backward_kernel<<<grid_for(V2 * c2), 256, 0, u->st>>>(g + G.gp2, c2, n2, g + G.gs2, 1);
  relu_b(g + G.gs2, a + A.a2b, V2 * c2);
  UN_CUDA(conv_back<T>(u, 3, a + A.a2a, c2, nullptr, 0, g + G.gs2, n2, g + G.ga2a, nullptr, 0));
  relu_b(g + G.ga2a, a + A.a2a, V2 * c2);
  UN_CUDA(conv_back<T>(u, 2, a + A.p1, c1, nullptr, 0, g + G.ga2a, n2, g + G.gp1, nullptr, 0));
  pool_backward_kernel<<<grid_for(V1 * c1), 256, 0, u->st>>>(g + G.gp1, c1, n, g + G.gs1, 1);
  relu_b(g + G.gs1, a + A.a1b, V1 * c1);
  UN_CUDA(conv_back<T>(u, 1, a + A.a1a, c1, nullptr, 0, g + G.gs1, n, g + G.ga1a, nullptr, 0));
  relu_b(g + G.ga1a, a + A.a1a, V1 * c1);
  UN_CUDA(conv_back<T>(u, 0, a + A.x, u->cin, nullptr, 0, g + G.ga1a, n, nullptr, nullptr, 0));
  UN_CUDA(cudaGetLastError());
  if (loss) {
    UN_CUDA(cudaMemcpyAsync(loss, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->st));
    UN_CUDA(cudaStreamSynchronize(u->st));
  }
  return RECON_OK;
}

}  // namespace

extern "C" {

recon_status recon_unet_param_count(int c1, size_t* count) {
  if ((c1 != 8 && c1 != 16) || !count) return RECON_ERR_INVALID_ARG;
  recon_unet tmp;
  tmp.c1 = c1;
  make_spec(&tmp);
  *count = tmp.np;
  return RECON_OK;
}

recon_status recon_unet_create(int c1, int bf16_storage, void* stream, recon_unet** out) {
  if (!out || (c1 != 8 && c1 != 16)) return RECON_ERR_INVALID_ARG;
  *out = nullptr;
  recon_unet* u = new recon_unet();
  u->c1 = c1;
  u->bf16 = bf16_storage ? 1 : 0;
  u->st = (cudaStream_t)stream;
  make_spec(u);
  const size_t es = u->bf16 ? 2 : 4;
  if (cudaMalloc(&u->p, u->np * 4) != cudaSuccess || cudaMalloc(&u->g, u->np * 4) != cudaSuccess ||
      cudaMalloc(&u->m1, u->np * 4) != cudaSuccess || cudaMalloc(&u->m2, u->np * 4) != cudaSuccess ||
      cudaMalloc(&u->decay, u->np) != cudaSuccess || cudaMalloc(&u->pt, u->np * es) != cudaSuccess ||
      cudaMalloc(&u->loss, sizeof(double)) != cudaSuccess || cudaMalloc(&u->dev_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    recon_unet_destroy(u);
    return RECON_ERR_OOM;
  }
  std::vector<unsigned char> dec(u->np, 0);
  for (size_t l = 0; l < u->spec.size(); ++l)
    for (size_t i = u->woff[l]; i < u->boff[l]; ++i) dec[i] = 1;
  if (cudaMemcpy(u->decay, dec.data(), u->np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(u->p, 0, u->np * 4) != cudaSuccess || cudaMemset(u->pt, 0, u->np * es) != cudaSuccess ||
      cudaMemset(u->m1, 0, u->np * 4) != cudaSuccess || cudaMemset(u->m2, 0, u->np * 4) != cudaSuccess ||
      cudaMemset(u->dev_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    recon_unet_destroy(u);
    return RECON_ERR_CUDA;
  }
  *out = u;
  return RECON_OK;
}

recon_status recon_unet_set_params(recon_unet* u, const float* host, size_t count) {
  if (!u || !host || count != u->np) return RECON_ERR_INVALID_ARG;
  UN_CUDA(cudaMemcpyAsync(u->p, host, u->np * 4, cudaMemcpyHostToDevice, u->st));
  if (u->bf16)
    to_t_kernel<bf16><<<grid_for((long long)u->np), 256, 0, u->st>>>(u->p, static_cast<bf16*>(u->pt), (long long)u->np);
  else
    UN_CUDA(cudaMemcpyAsync(u->pt, u->p, u->np * 4, cudaMemcpyDeviceToDevice, u->st));
  UN_CUDA(cudaMemsetAsync(u->m1, 0, u->np * 4, u->st));
  UN_CUDA(cudaMemsetAsync(u->m2, 0, u->np * 4, u->st));
  u->step = 0;
  ++u->pver;
  UN_CUDA(cudaStreamSynchronize(u->st));
  return RECON_OK;
}

recon_status recon_unet_get_params(recon_unet* u, float* host, size_t count) {
  if (!u || !host || count != u->np) return RECON_ERR_INVALID_ARG;
  UN_CUDA(cudaMemcpyAsync(host, u->p, u->np * 4, cudaMemcpyDeviceToHost, u->st));
  UN_CUDA(cudaStreamSynchronize(u->st));
  return RECON_OK;
}

recon_status recon_unet_get_grads(recon_unet* u, float* host, size_t count) {
  if (!u || !host || count != u->np) return RECON_ERR_INVALID_ARG;
  UN_CUDA(cudaMemcpyAsync(host, u->g, u->np * 4, cudaMemcpyDeviceToHost, u->st));
  UN_CUDA(cudaStreamSynchronize(u->st));
  return RECON_OK;
}

recon_status recon_unet_forward(recon_unet* u, const float* x, int n, float* y) {
  if (!u || !x || !y) return RECON_ERR_INVALID_ARG;
  recon_status rs = ensure(u, n, false);
  if (rs != RECON_OK) return rs;
  u->last_n = n;
  u->head_fused = false;
  if (u->bf16 && u->use_tc) return forward_tc(u, x, n, y);
  return u->bf16 ? forward_t<bf16>(u, x, n, y) : forward_t<float>(u, x, n, y);
}

recon_status recon_unet_backward(recon_unet* u, const float* x, const float* target, int n, double* loss) {
  if (!u || !x || !target) return RECON_ERR_INVALID_ARG;
  recon_status rs = ensure(u, n, true);
  if (rs != RECON_OK) return rs;
  u->last_n = n;
  u->head_fused = false;
  return u->bf16 ? backward_t<bf16>(u, x, target, n, loss) : backward_t<float>(u, x, target, n, loss);
}

recon_status recon_unet_adamw(recon_unet* u, float lr, float wd) {
  if (!u || !(lr > 0) || !(wd >= 0)) return RECON_ERR_INVALID_ARG;
  u->step += 1;
  ++u->pver;
  const float c1 = 1.f - powf(0.9f, (float)u->step), c2 = 1.f - powf(0.999f, (float)u->step);
  if (u->bf16)
    adamw_kernel<bf16><<<grid_for((long long)u->np), 256, 0, u->st>>>(u->p, u->g, u->m1, u->m2, u->decay,
                                                                       static_cast<bf16*>(u->pt), (long long)u->np, lr,
                                                                       wd, c1, c2);
  else
    adamw_kernel<float><<<grid_for((long long)u->np), 256, 0, u->st>>>(u->p, u->g, u->m1, u->m2, u->decay,
                                                                        static_cast<float*>(u->pt), (long long)u->np, lr,
                                                                        wd, c1, c2);
  UN_CUDA(cudaGetLastError());
  return RECON_OK;
}

recon_status recon_unet_destroy(recon_unet* u) {
  if (!u) return RECON_OK;
  if (u->st) cudaStreamSynchronize(u->st);
  cudaFree(u->p);
  cudaFree(u->g);
  cudaFree(u->m1);
  cudaFree(u->m2);
  cudaFree(u->decay);
  cudaFree(u->pt);
  cudaFree(u->loss);
  cudaFree(u->acts);
  cudaFree(u->grads);
  cudaFree(u->y);
  cudaFree(u->dev_err);
  cudaFree(u->wpack);
  delete u;
  return RECON_OK;
}

recon_status recon_unet_set_option(recon_unet* u, int option, int value) {
  if (!u) return RECON_ERR_INVALID_ARG;
  if (option == RECON_UNET_OPT_TENSOR_CORES) {
    u->use_tc = value ? 1 : 0;
    return RECON_OK;
  }
  return RECON_ERR_INVALID_ARG;
}

recon_status recon_unet_launch_count(recon_unet* u, long long* count) {
  if (!u || !count) return RECON_ERR_INVALID_ARG;
  *count = u->launches;
  return RECON_OK;
}

recon_status recon_unet_get_layer(recon_unet* u, int layer, float* host, size_t count) {
  if (!u || !host || layer < 0 || layer > 9 || !u->last_n || !u->acts) return RECON_ERR_INVALID_ARG;
  if (layer == 9 && u->head_fused) return RECON_ERR_STATE;
  static const int level[10] = {0, 0, 1, 1, 2, 2, 1, 1, 0, 0};
  const long long side = u->last_n >> level[layer];
  const size_t m = (size_t)(side * side * side) * u->spec[layer].cout;
  if (count != m) return RECON_ERR_INVALID_ARG;
  const Acts A = act_layout(u, u->last_n);
  const size_t offs[10] = {A.a1a, A.a1b, A.a2a, A.a2b, A.a3a, A.a3b, A.d2a, A.d2b, A.d1a, A.d1b};
  UN_CUDA(cudaStreamSynchronize(u->st));
  if (u->bf16) {
    std::vector<unsigned short> raw(m);
    UN_CUDA(cudaMemcpy(raw.data(), static_cast<const bf16*>(u->acts) + offs[layer], m * 2, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < m; ++i) {
      const unsigned int bits = (unsigned int)raw[i] << 16;
      std::memcpy(host + i, &bits, 4);
    }
  } else {
    UN_CUDA(cudaMemcpy(host, static_cast<const float*>(u->acts) + offs[layer], m * 4, cudaMemcpyDeviceToHost));
  }
  return RECON_OK;
}

const char* recon_unet_last_error(recon_unet* u) { return u ? u->err.c_str() : ""; }

}  // extern "C"
