// fft_core.cuh: shared-memory Stockham FFT building blocks for the reconstruction passes.
//
// A batch of complex lines of length L sits in shared memory; every stage of radix R reads R values
// at stride L/R, applies the inter-stage twiddles, does an R-point DFT in registers and writes the
// results in the autosorted (Stockham) order, so the output comes out in natural order with no bit
// reversal.  Mixed radices (2, 3, 4, 6, 8) give every mesh side 2^a 3^b used by the library.
// Transforms are unnormalised in both directions; the 1/N^3 of the inverse is applied once in
// the k-space kernels.  Twiddles come from a float32 table of exp(-2 pi i m / M) that the host
// computes in float64, so no fast-math sin/cos enters the transform.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Radix order of the plans of the mesh sides that have two (see the plan table at the end): 0 the
// default, largest radix first; 1 the alternative, smallest radix first.  A translation unit
// compiles one order, and its kernels live in that order's inline namespace, so the kernels of
// both orders link into one library under distinct names.
#ifndef RG_RADIX_ORDER
#define RG_RADIX_ORDER 0
#endif
#if RG_RADIX_ORDER == 0
#define RG_KNS order0
#else
#define RG_KNS order1
#endif

namespace rg {
inline namespace RG_KNS {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by i
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }

// ----------------------------------------------------------------------------------------------
// Small DFTs in registers.  Forward: y_m = sum_r x_r exp(-2 pi i r m / R); INV flips the sign.
// ----------------------------------------------------------------------------------------------
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct Dft<8, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float h = 0.70710678118654752f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    // o[m] *= w8^m, w8 = exp(-+ 2 pi i / 8)
    float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                    : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    float2 o2 = rot<INV>(o[2]);
    float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                    : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <bool INV>
struct Dft<3, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float s3 = 0.86602540378443865f;
    float2 a = v[0], b = v[1], c = v[2];
    float2 sum = cadd(b, c);
    float2 t = make_float2(a.x - 0.5f * sum.x, a.y - 0.5f * sum.y);
    float2 d = csub(b, c);
    // s = (b - c) * (-+ i sqrt(3)/2)
    float2 s = INV ? make_float2(-s3 * d.y, s3 * d.x) : make_float2(s3 * d.y, -s3 * d.x);
    v[0] = cadd(a, sum);
    v[1] = cadd(t, s);
    v[2] = csub(t, s);
  }
};

template <bool INV>
struct Dft<6, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float s3 = 0.86602540378443865f;
    float2 e[3] = {v[0], v[2], v[4]};
    float2 o[3] = {v[1], v[3], v[5]};
    Dft<3, INV>::run(e);
    Dft<3, INV>::run(o);
    // w6 = exp(-+ i pi / 3) = (1/2, -+ s3); w6^2 = (-1/2, -+ s3)
    const float sg = INV ? s3 : -s3;
    float2 o1 = cmul(o[1], make_float2(0.5f, sg));
    float2 o2 = cmul(o[2], make_float2(-0.5f, sg));
    v[0] = cadd(e[0], o[0]);
    v[3] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[4] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[5] = csub(e[2], o2);
  }
};

// ----------------------------------------------------------------------------------------------
// Shared-memory layouts.  Element i of line col lives at phys(i, col).  The swizzles make every
// Stockham access pattern (contiguous reads j + r L/R, strided first-stage writes 8 j + r) hit
// distinct banks within each 128-byte wavefront, with no padding.
//   ColLayout<C>: lines are the C columns of an [L][C] tile (strided passes); rows 8 apart that a
//                 wavefront touches together are moved to different bank halves by XOR-ing the
//                 row's low bits with bits 3.. of the row index.
//   RowLayout<L>: lines are rows (one per component); within each aligned 16-element block,
//                 bits 0-3 are XOR-ed with bits 3-6 (a permutation of the block).
// ----------------------------------------------------------------------------------------------
template <int C>
struct ColLayout {
  static constexpr bool kColFast = true;
  static constexpr int kMask = (C >= 16) ? 0 : (16 / C - 1);
  __device__ __forceinline__ static int phys(int i, int col) { return (i ^ ((i >> 3) & kMask)) * C + col; }
};

template <int L>
struct RowLayout {
  static constexpr bool kColFast = false;
  static constexpr int kStride = L;
  __device__ __forceinline__ static int phys(int i, int col) {
    return col * kStride + (i ^ ((i >> 3) & 15));
  }
};

// One Stockham stage over NCOL lines of length L with T threads.  The twiddle table holds
// exp(-2 pi i m / (L * TWS)); index m * TWS gives exp(-2 pi i m / L).  WARP selects a single warp
// working on its own lines (lane index, __syncwarp) instead of the whole CTA (__syncthreads).
template <bool WARP>
__device__ __forceinline__ int group_tid() { return WARP ? (threadIdx.x & 31) : threadIdx.x; }
template <bool WARP>
__device__ __forceinline__ void group_sync() {
  if (WARP) __syncwarp(); else __syncthreads();
}

// Stage twiddle tables.  A stage of radix R after NS points have been combined needs
// w^(r k) = exp(-2 pi i r k / (NS R)) for r = 1..R-1, k = 0..NS-1; they are stored per stage as
// [r - 1][k], so lanes with consecutive k read consecutive words.  OFF is the stage's offset in the
// table of the whole plan.
template <int L, int NCOL, int T, int R, int NS, int OFF, bool INV, class Lay, bool WARP>
__device__ __forceinline__ void stockham_stage(float2* __restrict__ s, const float2* __restrict__ tab) {
  constexpr int NBL = L / R;
  constexpr int NB = NBL * NCOL;
  constexpr int PER = (NB + T - 1) / T;
  const int tid = group_tid<WARP>();
  float2 v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = tid + p * T;
    if ((NB % T == 0) || b < NB) {
      const int col = Lay::kColFast ? (b % NCOL) : (b / NBL);
      const int j = Lay::kColFast ? (b / NCOL) : (b % NBL);
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = s[Lay::phys(j + r * NBL, col)];
      if (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tab[OFF + (r - 1) * NS + k];
          if (INV) w.y = -w.y;
          v[p][r] = cmul(v[p][r], w);
        }
      }
      Dft<R, INV>::run(v[p]);
    }
  }
  group_sync<WARP>();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = tid + p * T;
    if ((NB % T == 0) || b < NB) {
      const int col = Lay::kColFast ? (b % NCOL) : (b / NBL);
      const int j = Lay::kColFast ? (b / NCOL) : (b % NBL);
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[Lay::phys(base + r * NS, col)] = v[p][r];
    }
  }
  group_sync<WARP>();
}

template <int NS, int R>
constexpr int stage_tab_size() { return NS > 1 ? (R - 1) * NS : 0; }

template <int L, int NCOL, int T, bool INV, class Lay, bool WARP, int NS, int OFF, int R, int... Rest>
__device__ __forceinline__ void stockham_run(float2* s, const float2* tab) {
  stockham_stage<L, NCOL, T, R, NS, OFF, INV, Lay, WARP>(s, tab);
  if constexpr (sizeof...(Rest) > 0)
    stockham_run<L, NCOL, T, INV, Lay, WARP, NS * R, OFF + stage_tab_size<NS, R>(), Rest...>(s, tab);
}

// Fill the stage tables of a plan from the base table tw[m] = exp(-2 pi i m / (L TWS)).
template <int L, int TWS, int NS, int OFF, int R, int... Rest>
__device__ __forceinline__ void stockham_fill(float2* tab, const float2* tw, int tid, int nthr) {
  if (NS > 1) {
    constexpr int STEP = L / (NS * R);
    for (int e = tid; e < (R - 1) * NS; e += nthr) {
      const int r = 1 + e / NS, k = e % NS;
      tab[OFF + e] = tw[(r * k * STEP) * TWS];
    }
  }
  if constexpr (sizeof...(Rest) > 0) stockham_fill<L, TWS, NS * R, OFF + stage_tab_size<NS, R>(), Rest...>(tab, tw, tid, nthr);
}

template <int NS, int R, int... Rest>
constexpr int plan_tab_size() {
  if constexpr (sizeof...(Rest) > 0) return stage_tab_size<NS, R>() + plan_tab_size<NS * R, Rest...>();
  else return stage_tab_size<NS, R>();
}

// Radix plan per line length.
template <int L>
struct Plan;
#define RG_PLAN(LEN, ...)                                                                   \
  template <>                                                                               \
  struct Plan<LEN> {                                                                        \
    static constexpr int kTab = plan_tab_size<1, __VA_ARGS__>();                            \
    template <int NCOL, int T, bool INV, class Lay, bool WARP = false>                      \
    __device__ __forceinline__ static void run(float2* s, const float2* tab) {              \
      stockham_run<LEN, NCOL, T, INV, Lay, WARP, 1, 0, __VA_ARGS__>(s, tab);               \
    }                                                                                       \
    template <int TWS>                                                                      \
    __device__ __forceinline__ static void fill(float2* tab, const float2* tw, int tid, int nthr) { \
      stockham_fill<LEN, TWS, 1, 0, __VA_ARGS__>(tab, tw, tid, nthr);                      \
    }                                                                                       \
  };
RG_PLAN(16, 4, 4)
RG_PLAN(24, 8, 3)
RG_PLAN(32, 8, 4)
RG_PLAN(48, 8, 6)
RG_PLAN(64, 8, 8)
RG_PLAN(96, 8, 4, 3)
#if RG_RADIX_ORDER == 0
RG_PLAN(128, 8, 4, 4)
RG_PLAN(192, 8, 8, 3)
RG_PLAN(256, 8, 8, 4)
RG_PLAN(384, 8, 8, 6)
#else   // the 256 and 384 meshes (and their half-length z plans) smallest radix first
RG_PLAN(128, 4, 4, 8)
RG_PLAN(192, 3, 8, 8)
RG_PLAN(256, 4, 8, 8)
RG_PLAN(384, 6, 8, 8)
#endif
RG_PLAN(512, 8, 8, 8)
RG_PLAN(1024, 8, 8, 4, 4)
#undef RG_PLAN

}  // namespace RG_KNS
}  // namespace rg
