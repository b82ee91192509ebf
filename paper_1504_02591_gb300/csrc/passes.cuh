// passes.cuh: the three kinds of FFT pass of the reconstruction, each with its pointwise work fused.
//
// A 3-D r2c transform is three passes over the field: Z (contiguous rows, real <-> half complex),
// Y and X (strided lines, one [N x C] tile of C adjacent columns per CTA).  Work that is pointwise
// in configuration space rides on the Z pass (delta formation, the radial projection (Psi.r)r of
// Eq. Nusser); work that is pointwise in Fourier space rides on the X pass, between its forward
// and inverse transforms (Z[s] = i k s / k^2 of Eq. Zeldovich, the source update of Eq. iterative
// with its convergence norms).
#pragma once
#include <cuda.h>

#include "fft_core.cuh"
#include "types.h"

namespace rg {
inline namespace RG_KNS {   // the radix order's namespace (fft_core.cuh)

constexpr int kZThreads = 256;

// columns of one N = 512 k-space (y) tile: 4 adjacent kz (one 32-byte sector per row)
#ifndef RECON_KITER_COLS
#define RECON_KITER_COLS 4
#endif
template <int N, int MODE = 0, int NARROW = 0>
struct SCols {  // adjacent columns in one strided tile (the 3-component k-space tiles are narrower)
  static constexpr bool kK = (MODE == S_DELTA || MODE == S_ITER);
  static constexpr int kWide = ((N / 2) % 16 == 0 && N < 1024 && !NARROW) ? 16 : 8;   // must divide N / 2
  static constexpr int v = kK ? (N == 512 ? RECON_KITER_COLS : 4) : kWide;
  static_assert((N / 2) % v == 0 && N % v == 0, "tile columns must divide the half-grid rows");
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;  // valid in thread 0
}

// ------------------------------------------------------------------------------------------------
// Z pass: real rows of N floats <-> N/2+1 complex values (kz = 0..N/2).
// A real row is packed as N/2 complex z_m = x_2m + i x_2m+1 and transformed with an N/2-point FFT;
// the split into even/odd spectra with the exp(-2 pi i k / N) twiddles completes the r2c (and the
// reverse for c2r, which returns N times the inverse transform of the row).
// Each warp owns one row (all of its components) at a time and synchronises only with itself, so
// the CTA never waits at a block-wide barrier inside the row loop.
// ------------------------------------------------------------------------------------------------
template <int N, int NCOL>
__device__ __forceinline__ void r2c_split(float2* s, float2* qv, const float2* tw, int lane) {
  constexpr int L = N / 2;
  using Lay = RowLayout<L>;
  // every line: pairs (k, L - k) for k = 1..L/2, and k = 0 (which also gives the Nyquist value)
  for (int e = lane; e < NCOL * (L / 2 + 1); e += 32) {
    const int col = e / (L / 2 + 1), k = e % (L / 2 + 1);
    if (k == 0) {
      float2 z0 = s[Lay::phys(0, col)];
      s[Lay::phys(0, col)] = make_float2(z0.x + z0.y, 0.f);
      qv[col] = make_float2(z0.x - z0.y, 0.f);
    } else {
      const float2 zk = s[Lay::phys(k, col)], zm = s[Lay::phys(L - k, col)];
      const float2 wk = tw[k], wm = tw[L - k];
      // X[k] = (Zk + conj Zm)/2 - i w^k (Zk - conj Zm)/2
      float2 ev = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      float2 o = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));
      float2 xk = cadd(ev, cmul(make_float2(o.y, -o.x), wk));
      float2 ev2 = make_float2(0.5f * (zm.x + zk.x), 0.5f * (zm.y - zk.y));
      float2 o2 = make_float2(0.5f * (zm.x - zk.x), 0.5f * (zm.y + zk.y));
      float2 xm = cadd(ev2, cmul(make_float2(o2.y, -o2.x), wm));
      s[Lay::phys(k, col)] = xk;
      s[Lay::phys(L - k, col)] = xm;
    }
  }
}

template <int N, int NCOL>
__device__ __forceinline__ void c2r_merge(float2* s, const float2* qv, const float2* tw, int lane) {
  constexpr int L = N / 2;
  using Lay = RowLayout<L>;
  for (int e = lane; e < NCOL * (L / 2 + 1); e += 32) {
    const int col = e / (L / 2 + 1), k = e % (L / 2 + 1);
    if (k == 0) {
      const float2 x0 = s[Lay::phys(0, col)], xl = qv[col];
      // E = X0 + conj XL, O = X0 - conj XL, Z0 = E + i O
      float2 ev = make_float2(x0.x + xl.x, x0.y - xl.y);
      float2 o = make_float2(x0.x - xl.x, x0.y + xl.y);
      s[Lay::phys(0, col)] = cadd(ev, mul_i(o));
    } else {
      const float2 xk = s[Lay::phys(k, col)], xm = s[Lay::phys(L - k, col)];
      const float2 wk = cconj(tw[k]), wm = cconj(tw[L - k]);
      float2 ev = make_float2(xk.x + xm.x, xk.y - xm.y);
      float2 o = cmul(make_float2(xk.x - xm.x, xk.y + xm.y), wk);
      float2 ev2 = make_float2(xm.x + xk.x, xm.y - xk.y);
      float2 o2 = cmul(make_float2(xm.x - xk.x, xm.y + xk.y), wm);
      s[Lay::phys(k, col)] = cadd(ev, mul_i(o));
      s[Lay::phys(L - k, col)] = cadd(ev2, mul_i(o2));
    }
  }
}

constexpr int kZWarps = kZThreads / 32;

template <int N, int MODE>
struct ZWarpSmem {  // float2 slots of one warp's private region
  static constexpr int NF = (MODE == Z_DELTA) ? 1 : 3;
  static constexpr int kLines = (NF * RowLayout<N / 2>::kStride + 1) & ~1;   // even: keeps raw 16-B aligned
  static constexpr int kQ = 4;                                  // Nyquist values (padded)
  static constexpr int kRaw = (MODE == Z_DELTA) ? N : (MODE == Z_WARM ? N / 4 : 0);   // raw rows / coarse row
  static constexpr int v = kLines + kQ + kRaw + ((kLines + kQ + kRaw) & 1);
};

// 1024-point lines hold twice the butterflies per thread: two CTAs per SM (128 registers) there;
// the radix-3 and 64-point rows of N = 384 and 128 spill at 64 registers, so three CTAs (85)
template <int N>
constexpr int kZMinBlocks = N >= 1024 ? 2 : ((N == 384 || N == 128) ? 3 : 4);

template <int N, int MODE, int NC>
__global__ void __launch_bounds__(kZThreads, kZMinBlocks<N>) zpass_kernel(const ZArgs a) {
  constexpr int L = N / 2;
  constexpr int NF = (MODE == Z_DELTA) ? 1 : NC;   // lines transformed per row
  using Lay = RowLayout<L>;
  constexpr int WS = ZWarpSmem<N, MODE>::v;
  constexpr int TABZ = (Plan<L>::kTab + 1) & ~1;
  extern __shared__ float4 zsm[];
  float2* tw = reinterpret_cast<float2*>(zsm);                       // exp(-2 pi i k / N), k <= L
  float2* tab = tw + L + 2;                                          // stage twiddles of the L-point FFT
  float* taps = reinterpret_cast<float*>(tab + TABZ);                // N floats (Z_DELTA)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* s = tab + TABZ + N / 2 + warp * WS;                        // this warp's lines
  float2* qv = s + ZWarpSmem<N, MODE>::kLines;
  float* raw = reinterpret_cast<float*>(qv + ZWarpSmem<N, MODE>::kQ);
  __shared__ double red_sh[kZWarps];

  for (int m = threadIdx.x; m <= L; m += kZThreads) tw[m] = a.tw[m];
  for (int m = threadIdx.x; m < Plan<L>::kTab; m += kZThreads) tab[m] = a.tab[m];
  if (MODE == Z_DELTA)
    for (int j = threadIdx.x; j < a.ntap; j += kZThreads) taps[j] = a.taps[j];
  __syncthreads();

  float acc0 = 0.f, acc1 = 0.f;
  constexpr bool kInverse = (MODE == Z_INV || MODE == Z_PROJ || MODE == Z_FINAL || MODE == Z_RADIAL);
  // device-driven iteration: once the loop flag says converged, this pass writes the real Psi
  const bool fin = (MODE == Z_PROJ) && a.loop_flag && *a.loop_flag == 1;
  float inv_alpha = 0.f, thr = 0.f;
  const int nin = a.uniform ? 1 : 2;
  if (MODE == Z_DELTA) {
    const double* red = a.red;
    inv_alpha = a.uniform ? (float)((double)N * N * N / red[RED_SUM_WG]) : (float)(red[RED_SUM_WR] / red[RED_SUM_WG]);
    thr = a.uniform ? 0.f : (float)(a.mask_frac * red[RED_SUM_WR] / red[RED_CNT_RPOS]);
  }

  for (size_t row = (size_t)blockIdx.x * kZWarps + warp; row < (size_t)N * N; row += (size_t)gridDim.x * kZWarps) {
    if (kInverse) {
      // half-complex rows (L values) and Nyquist values of every component
      for (int e = lane; e < NC * (L / 2); e += 32) {
        const int q = e / (L / 2), m2 = e % (L / 2);
        const float4 v = reinterpret_cast<const float4*>(a.f[q].M + row * L)[m2];
        s[Lay::phys(2 * m2, q)] = make_float2(v.x, v.y);
        s[Lay::phys(2 * m2 + 1, q)] = make_float2(v.z, v.w);
      }
      if (lane < NC) qv[lane] = a.f[lane].Q[row];
      __syncwarp();
      if ((MODE == Z_PROJ || MODE == Z_RADIAL) && NC == 3 && !fin) {
        // the projection needs only C = dx Psi_x + dy Psi_y and Psi_z (dx and dy are constant along
        // the row), so two rows are transformed each way: C into line 0, Psi_z into line 1
        const Geometry& g = a.g;
        const float dx = g.los_mode == 1 ? g.los.x : g.off[row / N];
        const float dy = g.los_mode == 1 ? g.los.y : g.off[N + row % N];
        for (int m = lane; m < L; m += 32) {
          const float2 p0 = s[Lay::phys(m, 0)], p1 = s[Lay::phys(m, 1)], p2 = s[Lay::phys(m, 2)];
          s[Lay::phys(m, 0)] = make_float2(fmaf(dx, p0.x, dy * p1.x), fmaf(dx, p0.y, dy * p1.y));
          s[Lay::phys(m, 1)] = p2;
        }
        if (lane == 0) {
          const float2 q0 = qv[0], q1 = qv[1];
          qv[0] = make_float2(fmaf(dx, q0.x, dy * q1.x), fmaf(dx, q0.y, dy * q1.y));
          qv[1] = qv[2];
        }
        __syncwarp();
        c2r_merge<N, 2>(s, qv, tw, lane);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; ++q) Plan<L>::template run<1, 32, true, Lay, true>(s + q * Lay::kStride, tab);
      } else {
        c2r_merge<N, NF>(s, qv, tw, lane);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NF; ++q) Plan<L>::template run<1, 32, true, Lay, true>(s + q * Lay::kStride, tab);
      }
    } else if (MODE == Z_USTART || MODE == Z_WARM) {
      // a radial displacement u: P = u r on the row, then its forward r2c.  Z_WARM adds to
      // u the trilinear (periodic) upsampling of a coarse correction: the coarse node J of level l
      // sits at fine index (J + 1/2) 2^l - 1/2 along each axis.
      const Geometry& g = a.g;
      const int ix = (int)(row / N), iy = (int)(row % N);
      const float dx = g.los_mode == 1 ? 0.f : g.off[ix], dy = g.los_mode == 1 ? 0.f : g.off[N + iy];
      const float* ur = a.u_in + row * N;
      float* crow = raw;   // Z_WARM: the correction bilinearly interpolated to this (x, y) row
      int nc = 0, fl = 0;
      float inv_f = 0.f;
      if (MODE == Z_WARM) {
        fl = a.clevel;
        nc = N >> fl;
        inv_f = 1.f / (float)(1 << fl);
        const float tx = ((float)ix + 0.5f) * inv_f - 0.5f, ty = ((float)iy + 0.5f) * inv_f - 0.5f;
        const float fx = floorf(tx), fy = floorf(ty);
        const float wx = tx - fx, wy = ty - fy;
        int x0 = (int)fx, y0 = (int)fy;
        x0 = x0 < 0 ? x0 + nc : x0;
        y0 = y0 < 0 ? y0 + nc : y0;
        const int x1 = x0 + 1 == nc ? 0 : x0 + 1, y1 = y0 + 1 == nc ? 0 : y0 + 1;
        const size_t r00 = ((size_t)x0 * nc + y0) * nc, r01 = ((size_t)x0 * nc + y1) * nc;
        const size_t r10 = ((size_t)x1 * nc + y0) * nc, r11 = ((size_t)x1 * nc + y1) * nc;
        for (int j = lane; j < nc; j += 32) {
          const float c00 = a.corr[r00 + j] - a.ucoarse[r00 + j], c01 = a.corr[r01 + j] - a.ucoarse[r01 + j];
          const float c10 = a.corr[r10 + j] - a.ucoarse[r10 + j], c11 = a.corr[r11 + j] - a.ucoarse[r11 + j];
          crow[j] = (1.f - wx) * ((1.f - wy) * c00 + wy * c01) + wx * ((1.f - wy) * c10 + wy * c11);
        }
        __syncwarp();
      }
      for (int m = lane; m < L; m += 32) {
        float2 uu = reinterpret_cast<const float2*>(ur)[m];
        if (MODE == Z_WARM) {
          float add[2];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const float tz = ((float)(2 * m + h2) + 0.5f) * inv_f - 0.5f;
            const float fz = floorf(tz);
            const float wz = tz - fz;
            int z0 = (int)fz;
            z0 = z0 < 0 ? z0 + nc : z0;
            const int z1 = z0 + 1 == nc ? 0 : z0 + 1;
            add[h2] = (1.f - wz) * crow[z0] + wz * crow[z1];
          }
          uu.x += add[0];
          uu.y += add[1];
        }
        // P = u r = d psi with psi = w u (radial: w = 1/|d|; fixed LOS: d = the LOS, w = 1): line 0
        // takes psi, line 1 dz psi (the forward pass below writes dx psi^, dy psi^ and (dz psi)^)
        float dz0, dz1, w0, w1;
        if (g.los_mode == 1) {
          dz0 = dz1 = g.los.z;
          w0 = w1 = 1.f;
        } else {
          dz0 = g.off[2 * N + 2 * m];
          dz1 = g.off[2 * N + 2 * m + 1];
          const float q0 = fmaf(dx, dx, fmaf(dy, dy, dz0 * dz0));
          const float q1 = fmaf(dx, dx, fmaf(dy, dy, dz1 * dz1));
          w0 = q0 > 0.f ? rsqrtf(q0) : 0.f;
          w1 = q1 > 0.f ? rsqrtf(q1) : 0.f;
        }
        const float p0 = uu.x * w0, p1 = uu.y * w1;
        s[Lay::phys(m, 0)] = make_float2(p0, p1);
        s[Lay::phys(m, 1)] = make_float2(dz0 * p0, dz1 * p1);
      }
      __syncwarp();
    } else if (MODE == Z_DELTA) {
      // rows of rho_g (and rho_r) smoothed along x and y: z factor of the Gaussian as a periodic
      // convolution, then delta (Sec. 3.2) node by node
      for (int e = lane; e < nin * (N / 4); e += 32) {
        const int q = e / (N / 4), m4 = e % (N / 4);
        reinterpret_cast<float4*>(raw + q * N)[m4] = reinterpret_cast<const float4*>(a.f[q].M + row * L)[m4];
      }
      __syncwarp();
      const float* rg = raw;
      const float* rr = raw + N;
      for (int z = lane; z < N; z += 32) {
        int idx = z + a.t0;
        if (idx < 0) idx += N;
        float g = 0.f, r = 0.f;
        if (nin == 1) {
          for (int j = 0; j < a.ntap; ++j) {
            g = fmaf(taps[j], rg[idx], g);
            if (++idx == N) idx = 0;
          }
        } else {
          for (int j = 0; j < a.ntap; ++j) {
            g = fmaf(taps[j], rg[idx], g);
            r = fmaf(taps[j], rr[idx], r);
            if (++idx == N) idx = 0;
          }
        }
        // q = 1 + delta as the density ratio itself: the logarithm takes q, not 1 + (q - 1), which
        // in float32 would lose the digits of a low-density node to cancellation
        float q;
        if (nin == 1) {
          q = g * inv_alpha;
        } else {
          const bool in = r > thr;
          q = in ? g * inv_alpha / r : 1.f;
          acc1 += in ? 1.f : 0.f;
        }
        float d = q - 1.f;
        if (a.lognormal) {
          d = logf(fmaxf(q, 1e-6f));
          acc0 += d;
        }
        if (a.delta_real) a.delta_real[row * N + z] = d;
        reinterpret_cast<float*>(s + Lay::phys(z >> 1, 0))[z & 1] = d;
      }
      __syncwarp();
    } else {
      // real rows of N floats as L packed complex values
      for (int e = lane; e < NC * (L / 2); e += 32) {
        const int q = e / (L / 2), m2 = e % (L / 2);
        const float4 v = reinterpret_cast<const float4*>(a.f[q].M + row * L)[m2];
        s[Lay::phys(2 * m2, q)] = make_float2(v.x, v.y);
        s[Lay::phys(2 * m2 + 1, q)] = make_float2(v.z, v.w);
      }
      __syncwarp();
    }

    if (MODE == Z_RADIAL) {
      // s holds C and Psi_z (as in the projection): the start's radial displacement
      // u = coef w (C + dz Psi_z) = coef (Psi.r), as a real row
      const Geometry& g = a.g;
      const int ix = (int)(row / N), iy = (int)(row % N);
      const float dx = g.los_mode == 1 ? 0.f : g.off[ix], dy = g.los_mode == 1 ? 0.f : g.off[N + iy];
      for (int m = lane; m < L; m += 32) {
        const float2 c = s[Lay::phys(m, 0)], pz = s[Lay::phys(m, 1)];
        float dz0, dz1, w0, w1;
        if (g.los_mode == 1) {
          dz0 = dz1 = g.los.z;
          w0 = w1 = 1.f;
        } else {
          dz0 = g.off[2 * N + 2 * m];
          dz1 = g.off[2 * N + 2 * m + 1];
          const float q0 = fmaf(dx, dx, fmaf(dy, dy, dz0 * dz0));
          const float q1 = fmaf(dx, dx, fmaf(dy, dy, dz1 * dz1));
          w0 = q0 > 0.f ? rsqrtf(q0) : 0.f;
          w1 = q1 > 0.f ? rsqrtf(q1) : 0.f;
        }
        const float u0 = a.coef * (w0 * fmaf(dz0, pz.x, c.x));
        const float u1 = a.coef * (w1 * fmaf(dz1, pz.y, c.y));
        reinterpret_cast<float2*>(a.u_out + row * N)[m] = make_float2(u0, u1);
      }
      __syncwarp();
      continue;
    }

    if (MODE == Z_PROJ && NC == 3 && !fin) {
      // s holds C and Psi_z at z = 2m (.x) and 2m + 1 (.y); with r = w d (radial: w = 1/|d|; fixed
      // LOS: d = the LOS, w = 1), u = coef w (C + dz Psi_z) = coef (Psi.r) and P = u r = d psi with
      // psi = w u (Eq. Nusser): line 0 takes psi, line 1 dz psi
      const Geometry& g = a.g;
      const float dx = g.los_mode == 1 ? g.los.x : g.off[row / N];
      const float dy = g.los_mode == 1 ? g.los.y : g.off[N + row % N];
      for (int m = lane; m < L; m += 32) {
        const float2 c = s[Lay::phys(m, 0)], pz = s[Lay::phys(m, 1)];
        float dz0, dz1, w0, w1;
        if (g.los_mode == 1) {
          dz0 = dz1 = g.los.z;
          w0 = w1 = 1.f;
        } else {
          dz0 = g.off[2 * N + 2 * m];
          dz1 = g.off[2 * N + 2 * m + 1];
          const float q0 = fmaf(dx, dx, fmaf(dy, dy, dz0 * dz0));
          const float q1 = fmaf(dx, dx, fmaf(dy, dy, dz1 * dz1));
          w0 = q0 > 0.f ? rsqrtf(q0) : 0.f;
          w1 = q1 > 0.f ? rsqrtf(q1) : 0.f;
        }
        const float p0 = a.coef * (w0 * fmaf(dz0, pz.x, c.x)) * w0;
        const float p1 = a.coef * (w1 * fmaf(dz1, pz.y, c.y)) * w1;
        s[Lay::phys(m, 0)] = make_float2(p0, p1);
        s[Lay::phys(m, 1)] = make_float2(dz0 * p0, dz1 * p1);
      }
      __syncwarp();
    } else if (MODE == Z_PROJ && !fin) {
      // s holds Psi_j(x, y, z), z = 2m (.x) and 2m + 1 (.y): P = coef (Psi.r) r (Eq. Nusser)
      const Geometry& g = a.g;
      const int ix = (int)(row / N), iy = (int)(row % N);
      float dx = 0.f, dy = 0.f;
      if (g.los_mode != 1) {
        dx = g.off[ix];
        dy = g.off[N + iy];
      }
      for (int m = lane; m < L; m += 32) {
        const float2 p0 = s[Lay::phys(m, 0)], p1 = s[Lay::phys(m, 1)], p2 = s[Lay::phys(m, 2)];
        float rx0, ry0, rz0, rx1, ry1, rz1;
        if (g.los_mode == 1) {
          rx0 = rx1 = g.los.x; ry0 = ry1 = g.los.y; rz0 = rz1 = g.los.z;
        } else {
          const float dz0 = g.off[2 * N + 2 * m], dz1 = g.off[2 * N + 2 * m + 1];
          const float q0 = fmaf(dx, dx, fmaf(dy, dy, dz0 * dz0));
          const float q1 = fmaf(dx, dx, fmaf(dy, dy, dz1 * dz1));
          const float i0 = q0 > 0.f ? rsqrtf(q0) : 0.f;
          const float i1 = q1 > 0.f ? rsqrtf(q1) : 0.f;
          rx0 = dx * i0; ry0 = dy * i0; rz0 = dz0 * i0;
          rx1 = dx * i1; ry1 = dy * i1; rz1 = dz1 * i1;
        }
        const float u0 = a.coef * fmaf(p0.x, rx0, fmaf(p1.x, ry0, p2.x * rz0));
        const float u1 = a.coef * fmaf(p0.y, rx1, fmaf(p1.y, ry1, p2.y * rz1));
        s[Lay::phys(m, 0)] = make_float2(u0 * rx0, u1 * rx1);
        s[Lay::phys(m, 1)] = make_float2(u0 * ry0, u1 * ry1);
        s[Lay::phys(m, 2)] = make_float2(u0 * rz0, u1 * rz1);
      }
      __syncwarp();
    }

    if (MODE == Z_INV || MODE == Z_FINAL || (MODE == Z_PROJ && fin)) {
      for (int e = lane; e < NC * (L / 2); e += 32) {
        const int q = e / (L / 2), m2 = e % (L / 2);
        const float2 v0 = s[Lay::phys(2 * m2, q)], v1 = s[Lay::phys(2 * m2 + 1, q)];
        reinterpret_cast<float4*>(a.f[q].M + row * L)[m2] = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    } else if ((MODE == Z_PROJ || MODE == Z_USTART || MODE == Z_WARM) && NC == 3) {
      // psi^ and (dz psi)^; P_x = dx psi^ and P_y = dy psi^ are scaled copies
#pragma unroll
      for (int q = 0; q < 2; ++q) Plan<L>::template run<1, 32, false, Lay, true>(s + q * Lay::kStride, tab);
      r2c_split<N, 2>(s, qv, tw, lane);
      __syncwarp();
      const Geometry& g = a.g;
      const float dx = g.los_mode == 1 ? g.los.x : g.off[row / N];
      const float dy = g.los_mode == 1 ? g.los.y : g.off[N + row % N];
      for (int m2 = lane; m2 < L / 2; m2 += 32) {
        const float2 v0 = s[Lay::phys(2 * m2, 0)], v1 = s[Lay::phys(2 * m2 + 1, 0)];
        const float2 z0 = s[Lay::phys(2 * m2, 1)], z1 = s[Lay::phys(2 * m2 + 1, 1)];
        reinterpret_cast<float4*>(a.f[0].M + row * L)[m2] = make_float4(dx * v0.x, dx * v0.y, dx * v1.x, dx * v1.y);
        reinterpret_cast<float4*>(a.f[1].M + row * L)[m2] = make_float4(dy * v0.x, dy * v0.y, dy * v1.x, dy * v1.y);
        reinterpret_cast<float4*>(a.f[2].M + row * L)[m2] = make_float4(z0.x, z0.y, z1.x, z1.y);
      }
      if (lane == 0) {
        a.f[0].Q[row] = cscale(qv[0], dx);
        a.f[1].Q[row] = cscale(qv[0], dy);
        a.f[2].Q[row] = qv[1];
      }
    } else {
#pragma unroll
      for (int q = 0; q < NF; ++q) Plan<L>::template run<1, 32, false, Lay, true>(s + q * Lay::kStride, tab);
      r2c_split<N, NF>(s, qv, tw, lane);
      __syncwarp();
      for (int e = lane; e < NF * (L / 2); e += 32) {
        const int q = e / (L / 2), m2 = e % (L / 2);
        const float2 v0 = s[Lay::phys(2 * m2, q)], v1 = s[Lay::phys(2 * m2 + 1, q)];
        float2* dst = (MODE == Z_DELTA) ? a.dout.M : a.f[q].M;
        reinterpret_cast<float4*>(dst + row * L)[m2] = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
      if (lane < NF) ((MODE == Z_DELTA) ? a.dout.Q : a.f[lane].Q)[row] = qv[lane];
    }
    __syncwarp();   // the stores above read s before the next row overwrites it
  }

  if (MODE == Z_DELTA) {
    double r0 = block_sum((double)acc0, red_sh);
    double r1 = block_sum((double)acc1, red_sh);
    if (threadIdx.x == 0) {
      a.partials[2 * blockIdx.x + 0] = r0;
      a.partials[2 * blockIdx.x + 1] = r1;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// The projection pass for N = 512 (rows of L = 256 complex values, radices 8 x 8 x 4), one warp per
// row.  Lane l holds the points l + 32 r (r = 0..7) of each component.  The c2r merge pairs point
// m with L - m, which for l >= 1 sits on lane 32 - l (lane 0 pairs with itself and the Nyquist
// value), so the merge runs on shuffles straight after the global loads and feeds the first
// inverse stage in registers.  The last inverse stage (radix 4, butterflies l and l + 32) leaves
// exactly the points l + 32 r on lane l, so the projection and the first forward stage run in
// registers too; the r2c split again pairs lanes l and 32 - l, and the results go straight to
// global memory.  Shared memory carries only the two middle stages of each transform.  The
// butterflies, twiddles and merge/split formulas are those of the generic pass.
// ------------------------------------------------------------------------------------------------
template <int N>
struct ZProj8 {
  static_assert(N == 512, "radices 8 x 8 x 4 of the 256-point row transform");
  static constexpr int L = N / 2;
  static constexpr int TABZ = (Plan<L>::kTab + 1) & ~1;
  static constexpr int kWarp = L + L / 2;      // FFT buffer + the coarse correction row (Z_WARM)
  static constexpr size_t smem = sizeof(float2) * ((size_t)L + 2 + TABZ + (size_t)kZWarps * kWarp);
};

// the middle stage (NS = 8, radix 8): butterfly l reads l + 32 r, writes (l / 8) 64 + l mod 8 + 8 r
template <bool INV>
__device__ __forceinline__ void zrow_mid(float2* __restrict__ s, const float2* __restrict__ tab, int lane) {
  using Lay = RowLayout<256>;
  float2 v[8];
  const int k = lane & 7;
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = s[Lay::phys(lane + 32 * r, 0)];
#pragma unroll
  for (int r = 1; r < 8; ++r) {
    float2 w = tab[(r - 1) * 8 + k];
    if (INV) w.y = -w.y;
    v[r] = cmul(v[r], w);
  }
  Dft<8, INV>::run(v);
  __syncwarp();
  const int base = (lane >> 3) * 64 + k;
#pragma unroll
  for (int r = 0; r < 8; ++r) s[Lay::phys(base + 8 * r, 0)] = v[r];
  __syncwarp();
}

// One 256-point transform: in, z[l + 32 r] (registers, r = 0..7); out, Z[j + 64 r] for the two
// butterflies j = l (A[r]) and j = l + 32 (B[r]), r = 0..3.
template <bool INV>
__device__ __forceinline__ void zrow_fft(float2 (&v)[8], float2 (&A)[4], float2 (&B)[4], float2* __restrict__ s,
                                         const float2* __restrict__ tab, int lane) {
  using Lay = RowLayout<256>;
  Dft<8, INV>::run(v);                                   // stage 1 (NS = 1): butterfly l, no twiddles
#pragma unroll
  for (int r = 0; r < 8; ++r) s[Lay::phys(8 * lane + r, 0)] = v[r];
  __syncwarp();
  zrow_mid<INV>(s, tab, lane);
#pragma unroll
  for (int h = 0; h < 2; ++h) {                          // stage 3 (NS = 64, radix 4): butterflies l, l + 32
    const int j = lane + 32 * h;
    float2 u[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) u[r] = s[Lay::phys(j + 64 * r, 0)];
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      float2 w = tab[56 + (r - 1) * 64 + j];
      if (INV) w.y = -w.y;
      u[r] = cmul(u[r], w);
    }
    Dft<4, INV>::run(u);
#pragma unroll
    for (int r = 0; r < 4; ++r) (h ? B : A)[r] = u[r];
  }
  __syncwarp();                                          // s is reused by the next line
}

// c2r of one component's row (loaded by zrow_load: X[l + 32 r] and the Nyquist value): merge with
// the mirror X[L - l - 32 r] (on lane 32 - l; lane 0 with itself and the Nyquist value), inverse
// transform; out A[r] = x[l + 64 r], B[r] = x[l + 32 + 64 r] (complex points = real pairs 2m, 2m + 1).
__device__ __forceinline__ void zrow_load(const Field& f, size_t row, int lane, float2 (&x)[8], float2& xl) {
  const float2* src = f.M + row * 256;
#pragma unroll
  for (int r = 0; r < 8; ++r) x[r] = src[lane + 32 * r];
  xl = f.Q[row];
}

__device__ __forceinline__ void zrow_c2r(const float2 (&x)[8], float2 xl, int lane, int partner,
                                         const float2* __restrict__ tw, float2* __restrict__ s,
                                         const float2* __restrict__ tab, float2 (&A)[4], float2 (&B)[4]) {
  float2 z[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    float2 xm;
    xm.x = __shfl_sync(0xffffffffu, x[7 - r].x, partner);
    xm.y = __shfl_sync(0xffffffffu, x[7 - r].y, partner);
    if (lane == 0) xm = (r == 0) ? xl : x[(8 - r) & 7];
    const float2 w = cconj(tw[lane + 32 * r]);
    const float2 xk = x[r];
    const float2 ev = make_float2(xk.x + xm.x, xk.y - xm.y);
    const float2 o = cmul(make_float2(xk.x - xm.x, xk.y + xm.y), w);
    z[r] = cadd(ev, mul_i(o));
  }
  zrow_fft<true>(z, A, B, s, tab, lane);
}

// r2c of one component's row from the real points v[r] = (x[2m], x[2m + 1]), m = l + 32 r: forward
// transform, split (pairs k, L - k on lanes l and 32 - l), store the half-complex row and Nyquist value.
__device__ __forceinline__ void zrow_r2c(float2 (&v)[8], const Field& f, size_t row, int lane, int partner,
                                         const float2* __restrict__ tw, float2* __restrict__ s,
                                         const float2* __restrict__ tab) {
  constexpr int L = 256;
  float2 Y0[4], Y1[4];
  zrow_fft<false>(v, Y0, Y1, s, tab, lane);
  float2* dst = f.M + row * L;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 pa, pb;
    pa.x = __shfl_sync(0xffffffffu, Y1[3 - r].x, partner);
    pa.y = __shfl_sync(0xffffffffu, Y1[3 - r].y, partner);
    pb.x = __shfl_sync(0xffffffffu, Y0[3 - r].x, partner);
    pb.y = __shfl_sync(0xffffffffu, Y0[3 - r].y, partner);
    if (lane == 0) {
      pa = Y0[(4 - r) & 3];
      pb = Y1[3 - r];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h + 64 * r;
      const float2 zk = h ? Y1[r] : Y0[r], zm = h ? pb : pa;
      float2 xk;
      if (k == 0) {
        xk = make_float2(zk.x + zk.y, 0.f);
        f.Q[row] = make_float2(zk.x - zk.y, 0.f);
      } else {
        const float2 ev = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 o = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));
        xk = cadd(ev, cmul(make_float2(o.y, -o.x), tw[k]));
      }
      dst[k] = xk;
    }
  }
}

// The observer offset d = (dx, dy, dz) of a node and w with r = w d the line of sight (radial: w =
// 1/|d|, zero at the observer; fixed LOS: d = the LOS vector, w = 1), at the real points 2m and
// 2m + 1 of a row; dx and dy are the row's.
__device__ __forceinline__ void zrow_dw(const Geometry& g, float dx, float dy, int m, float& dz0, float& dz1,
                                        float& w0, float& w1) {
  if (g.los_mode == 1) {
    dz0 = dz1 = g.los.z;
    w0 = w1 = 1.f;
    return;
  }
  const int n = g.n;
  dz0 = g.off[2 * n + 2 * m];
  dz1 = g.off[2 * n + 2 * m + 1];
  const float q0 = fmaf(dx, dx, fmaf(dy, dy, dz0 * dz0));
  const float q1 = fmaf(dx, dx, fmaf(dy, dy, dz1 * dz1));
  w0 = q0 > 0.f ? rsqrtf(q0) : 0.f;
  w1 = q1 > 0.f ? rsqrtf(q1) : 0.f;
}

// The z passes of the register-fused path, one warp per row.  With r = w d, the projection
// P = coef (Psi.r) r needs only C = dx Psi_x + dy Psi_y and Psi_z (dx, dy are constant along a z
// row, so C is formed before the transform):  u = coef w (C + dz Psi_z) and P_j = d_j psi with
// psi = w u.  So the pass transforms two rows each way and leaves psi^ = r2c(psi) and
// Z^ = r2c(dz psi) (P_x = dx psi^ and P_y = dy psi^ are formed by the forward x pass).
//   Z_PROJ:   c2r x2, P, r2c x2; once the device loop has converged, c2r x3 and the real Psi.
//             With a.cform (while the loop runs) C arrives formed in f[0] and Psi_z in wf.
//   Z_RADIAL: c2r x2, u as a real row (C form as Z_PROJ).
//   Z_WARM:   u from the real row plus the upsampled coarse correction, r2c x2.
//   Z_USTART: u from the real row, r2c x2.
template <int N, int MODE>
__global__ void __launch_bounds__(kZThreads, 2) zfused8_kernel(const ZArgs a) {
  constexpr int L = ZProj8<N>::L;
  extern __shared__ float4 zsm[];
  float2* tw = reinterpret_cast<float2*>(zsm);                        // exp(-2 pi i m / N), m <= L
  float2* tab = tw + L + 2;                                           // stage twiddles (256-point plan)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* s = tab + ZProj8<N>::TABZ + warp * ZProj8<N>::kWarp;
  float* crow = reinterpret_cast<float*>(s + L);                      // Z_WARM: this row's coarse correction
  for (int m = threadIdx.x; m <= L; m += kZThreads) tw[m] = a.tw[m];
  for (int m = threadIdx.x; m < Plan<L>::kTab; m += kZThreads) tab[m] = a.tab[m];
  __syncthreads();
  const bool fin = (MODE == Z_PROJ) && a.loop_flag && *a.loop_flag == 1;
  const int partner = (32 - lane) & 31;
  const Geometry& g = a.g;
  // rows (ix, iy) of every y-plane, or of the planes [ybeg, ybeg + ycount)
  const size_t nrows = a.ycount ? (size_t)N * a.ycount : (size_t)N * N;

  for (size_t lr = (size_t)blockIdx.x * kZWarps + warp; lr < nrows; lr += (size_t)gridDim.x * kZWarps) {
    const size_t row = a.ycount ? (lr / a.ycount) * N + a.ybeg + lr % a.ycount : lr;
    const int ix = (int)(row / N), iy = (int)(row % N);
    if (MODE == Z_PROJ && fin) {
      float2 x[3][8], xl[3], A[3][4], B[3][4];
#pragma unroll
      for (int q = 0; q < 3; ++q) zrow_load(a.f[q], row, lane, x[q], xl[q]);
#pragma unroll
      for (int q = 0; q < 3; ++q) zrow_c2r(x[q], xl[q], lane, partner, tw, s, tab, A[q], B[q]);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float2* dst = a.f[q].M + row * L;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          dst[lane + 64 * r] = A[q][r];
          dst[lane + 32 + 64 * r] = B[q][r];
        }
      }
      continue;
    }
    const float dx = g.los_mode == 1 ? g.los.x : g.off[ix], dy = g.los_mode == 1 ? g.los.y : g.off[N + iy];
    // the rows psi and dz psi at the points l + 64 r (A) and l + 32 + 64 r (B)
    float2 A[2][4], B[2][4];
    if (MODE == Z_WARM || MODE == Z_USTART) {
      float inv_f = 1.f, wx = 0.f, wy = 0.f;
      int nc = 1;
      if (MODE == Z_WARM) {
        // u = u_s + U[corr - ucoarse] (see the generic pass)
        const int fl = a.clevel;
        nc = N >> fl;
        inv_f = 1.f / (float)(1 << fl);
        const float tx = ((float)ix + 0.5f) * inv_f - 0.5f, ty = ((float)iy + 0.5f) * inv_f - 0.5f;
        const float fx = floorf(tx), fy = floorf(ty);
        wx = tx - fx;
        wy = ty - fy;
        int x0 = (int)fx, y0 = (int)fy;
        x0 = x0 < 0 ? x0 + nc : x0;
        y0 = y0 < 0 ? y0 + nc : y0;
        const int x1 = x0 + 1 == nc ? 0 : x0 + 1, y1 = y0 + 1 == nc ? 0 : y0 + 1;
        const size_t r00 = ((size_t)x0 * nc + y0) * nc, r01 = ((size_t)x0 * nc + y1) * nc;
        const size_t r10 = ((size_t)x1 * nc + y0) * nc, r11 = ((size_t)x1 * nc + y1) * nc;
        for (int jz = lane; jz < nc; jz += 32) {
          const float c00 = a.corr[r00 + jz] - a.ucoarse[r00 + jz], c01 = a.corr[r01 + jz] - a.ucoarse[r01 + jz];
          const float c10 = a.corr[r10 + jz] - a.ucoarse[r10 + jz], c11 = a.corr[r11 + jz] - a.ucoarse[r11 + jz];
          crow[jz] = (1.f - wx) * ((1.f - wy) * c00 + wy * c01) + wx * ((1.f - wy) * c10 + wy * c11);
        }
        __syncwarp();
      }
      const float2* ur = reinterpret_cast<const float2*>(a.u_in + row * N);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int m = lane + 32 * h + 64 * r;
          float2 uu = ur[m];
          if (MODE == Z_WARM) {
            float add[2];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const float tz = ((float)(2 * m + h2) + 0.5f) * inv_f - 0.5f;
              const float fz = floorf(tz);
              const float wz = tz - fz;
              int z0 = (int)fz;
              z0 = z0 < 0 ? z0 + nc : z0;
              const int z1 = z0 + 1 == nc ? 0 : z0 + 1;
              add[h2] = (1.f - wz) * crow[z0] + wz * crow[z1];
            }
            uu.x += add[0];
            uu.y += add[1];
          }
          float dz0, dz1, w0, w1;
          zrow_dw(g, dx, dy, m, dz0, dz1, w0, w1);
          const float p0 = uu.x * w0, p1 = uu.y * w1;
          (h ? B : A)[0][r] = make_float2(p0, p1);
          (h ? B : A)[1][r] = make_float2(dz0 * p0, dz1 * p1);
        }
      if (MODE == Z_WARM) __syncwarp();   // crow is rewritten by the next row
    } else {
      float2 x[3][8], xl[3];
      if ((MODE == Z_PROJ || MODE == Z_RADIAL) && a.cform) {   // C and Psi_z from the inverse x pass
        zrow_load(a.f[0], row, lane, x[0], xl[0]);
        zrow_load(a.wf, row, lane, x[2], xl[2]);
      } else {
        // all three rows' loads in flight before the first transform; C = dx Psi_x + dy Psi_y
#pragma unroll
        for (int q = 0; q < 3; ++q) zrow_load(a.f[q], row, lane, x[q], xl[q]);
#pragma unroll
        for (int r = 0; r < 8; ++r)
          x[0][r] = make_float2(fmaf(dx, x[0][r].x, dy * x[1][r].x), fmaf(dx, x[0][r].y, dy * x[1][r].y));
        xl[0] = make_float2(fmaf(dx, xl[0].x, dy * xl[1].x), fmaf(dx, xl[0].y, dy * xl[1].y));
      }
      zrow_c2r(x[0], xl[0], lane, partner, tw, s, tab, A[0], B[0]);
      zrow_c2r(x[2], xl[2], lane, partner, tw, s, tab, A[1], B[1]);
      // u = coef (Psi . r) at the real points 2m, 2m + 1 of the complex point m (Eq. Nusser)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int m = lane + 32 * h + 64 * r;
          float dz0, dz1, w0, w1;
          zrow_dw(g, dx, dy, m, dz0, dz1, w0, w1);
          const float2 c = h ? B[0][r] : A[0][r], pz = h ? B[1][r] : A[1][r];
          const float u0 = a.coef * (w0 * fmaf(dz0, pz.x, c.x));
          const float u1 = a.coef * (w1 * fmaf(dz1, pz.y, c.y));
          if (MODE == Z_RADIAL) {
            reinterpret_cast<float2*>(a.u_out + row * N)[m] = make_float2(u0, u1);
          } else {
            const float p0 = u0 * w0, p1 = u1 * w1;
            (h ? B : A)[0][r] = make_float2(p0, p1);
            (h ? B : A)[1][r] = make_float2(dz0 * p0, dz1 * p1);
          }
        }
      if (MODE == Z_RADIAL) continue;
    }
    {
      // the points l + 32 r of the real rows: A[r/2] (r even), B[(r-1)/2] (r odd)
      float2 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = (r & 1) ? B[0][r >> 1] : A[0][r >> 1];
      zrow_r2c(v, a.f[0], row, lane, partner, tw, s, tab);                      // psi^
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = (r & 1) ? B[1][r >> 1] : A[1][r >> 1];
      zrow_r2c(v, a.f[2], row, lane, partner, tw, s, tab);                      // Z^ = (dz psi)^
    }
  }
}

// Z_DELTA for N = 512 (at most 32 smoothing taps): each warp stages its row of rho_g (and rho_r)
// with the periodic continuation the z convolution reads, each lane convolves 16 consecutive nodes
// with the taps in registers (every staged value read once per 16 outputs; the row is stored with
// one pad word per 16 so the lanes' windows fall in distinct banks), forms delta (mask, lognormal)
// exactly as the generic pass, stores the real copy, and runs the r2c of the fused passes.
template <int N>
struct ZDelta8 {
  static_assert(N == 512, "rows of 256 complex points");
  static constexpr int L = N / 2, KT = 32, V = 16;
  static constexpr int kExt = N + KT + V;                       // staged entries per row
  static constexpr int kExtPad = kExt + kExt / 16 + 1;          // with one pad word per 16
  static constexpr int TABZ = (Plan<L>::kTab + 1) & ~1;
  static constexpr int kWarp = L + kExtPad;                      // float2: FFT buffer + two staged rows
  static constexpr size_t smem = sizeof(float2) * ((size_t)L + 2 + TABZ + (size_t)kZWarps * kWarp);
  __device__ __forceinline__ static int pad(int p) { return p + (p >> 4); }
};

template <int N>
__global__ void __launch_bounds__(kZThreads, 2) zdelta8_kernel(const ZArgs a) {
  using Z = ZDelta8<N>;
  constexpr int L = Z::L, KT = Z::KT, V = Z::V;
  using Lay = RowLayout<L>;
  extern __shared__ float4 zsm[];
  float2* tw = reinterpret_cast<float2*>(zsm);
  float2* tab = tw + L + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* s = tab + Z::TABZ + warp * Z::kWarp;
  float* xg = reinterpret_cast<float*>(s + L);                   // staged rho_g row, then rho_r row
  float* xr = xg + Z::kExtPad;
  __shared__ double red_sh[kZWarps];
  for (int m = threadIdx.x; m <= L; m += kZThreads) tw[m] = a.tw[m];
  for (int m = threadIdx.x; m < Plan<L>::kTab; m += kZThreads) tab[m] = a.tab[m];
  __syncthreads();
  float tp[KT];
#pragma unroll
  for (int jt = 0; jt < KT; ++jt) tp[jt] = jt < a.ntap ? a.taps[jt] : 0.f;
  const double* red = a.red;
  const int nin = a.uniform ? 1 : 2;
  const float inv_alpha = a.uniform ? (float)((double)N * N * N / red[RED_SUM_WG]) : (float)(red[RED_SUM_WR] / red[RED_SUM_WG]);
  const float thr = a.uniform ? 0.f : (float)(a.mask_frac * red[RED_SUM_WR] / red[RED_CNT_RPOS]);
  const int partner = (32 - lane) & 31;
  float acc0 = 0.f, acc1 = 0.f;

  for (size_t row = (size_t)blockIdx.x * kZWarps + warp; row < (size_t)N * N; row += (size_t)gridDim.x * kZWarps) {
    const float* rg = reinterpret_cast<const float*>(a.f[0].M) + row * N;
    const float* rr = reinterpret_cast<const float*>(a.f[1].M) + row * N;
    for (int p = lane; p < Z::kExt; p += 32) {
      int i = (p + a.t0) % N;
      if (i < 0) i += N;
      xg[Z::pad(p)] = rg[i];
      if (nin == 2) xr[Z::pad(p)] = rr[i];
    }
    __syncwarp();
    const int z0 = V * lane;
    float ag[V], ar[V];
#pragma unroll
    for (int v = 0; v < V; ++v) ag[v] = ar[v] = 0.f;
#pragma unroll
    for (int w = 0; w < KT + V - 1; ++w) {
      const float g = xg[Z::pad(z0 + w)];
      const float r = nin == 2 ? xr[Z::pad(z0 + w)] : 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int jt = w - v;
        if (jt >= 0 && jt < KT) {
          ag[v] = fmaf(tp[jt], g, ag[v]);
          if (nin == 2) ar[v] = fmaf(tp[jt], r, ar[v]);
        }
      }
    }
    float d[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float q;   // 1 + delta, kept as the ratio for the logarithm (see the generic pass)
      if (nin == 1) {
        q = ag[v] * inv_alpha;
      } else {
        const bool in = ar[v] > thr;
        q = in ? ag[v] * inv_alpha / ar[v] : 1.f;
        acc1 += in ? 1.f : 0.f;
      }
      float dv = q - 1.f;
      if (a.lognormal) {
        dv = logf(fmaxf(q, 1e-6f));
        acc0 += dv;
      }
      d[v] = dv;
    }
    if (a.delta_real) {
      float4* dr = reinterpret_cast<float4*>(a.delta_real + row * N + z0);
#pragma unroll
      for (int v4 = 0; v4 < V / 4; ++v4) dr[v4] = make_float4(d[4 * v4], d[4 * v4 + 1], d[4 * v4 + 2], d[4 * v4 + 3]);
    }
#pragma unroll
    for (int i = 0; i < V / 2; ++i) s[Lay::phys(z0 / 2 + i, 0)] = make_float2(d[2 * i], d[2 * i + 1]);
    __syncwarp();
    float2 v8[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v8[r] = s[Lay::phys(lane + 32 * r, 0)];
    __syncwarp();
    zrow_r2c(v8, a.dout, row, lane, partner, tw, s, tab);
  }
  const double r0 = block_sum((double)acc0, red_sh);
  const double r1 = block_sum((double)acc1, red_sh);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x + 0] = r0;
    a.partials[2 * blockIdx.x + 1] = r1;
  }
}

template <int N, int NC>
constexpr size_t zpass_smem(int mode) {
  return sizeof(float2) * ((size_t)N / 2 + 2 + ((Plan<N / 2>::kTab + 1) & ~1) + N / 2 +
                           (size_t)kZWarps * (mode == Z_DELTA  ? ZWarpSmem<N, Z_DELTA>::v
                                              : mode == Z_WARM ? ZWarpSmem<N, Z_WARM>::v
                                                               : ZWarpSmem<N, Z_PROJ>::v));
}

// ------------------------------------------------------------------------------------------------
// Strided passes (Y and X).  A tile is N lines x C adjacent columns.  Tiles over the main array M:
//   Y: lines along y at fixed x, columns kz0..kz0+C-1      (offset (x N + y) N/2 + kz)
//   X: lines along x at fixed ky, columns kz0..kz0+C-1     (offset (x N + ky) N/2 + kz)
// and over the Nyquist plane Q [kx][ky] (the k-space passes, which need all three components of
// P at once, run along y; the plain passes run along either axis):
//   Y: lines along y (contiguous), columns are C values of x
//   X: lines along x (stride N), columns are C adjacent ky
// ------------------------------------------------------------------------------------------------
struct Tile {
  size_t base;
  int ls, cs;      // line stride, column stride (complex elements)
  int isQ;
  int a;           // x (Y pass) or ky (X pass) of an M tile
  int c0;          // first kz (M) or first column (Q)
};

template <int N, int C, int AXIS>
__device__ __forceinline__ Tile tile_of(int t) {
  constexpr int H = N / 2;
  constexpr int MT = N * (H / C);
  Tile r;
  if (t < MT) {
    r.isQ = 0;
    r.a = t / (H / C);
    r.c0 = (t % (H / C)) * C;
    r.base = (AXIS == AX_Y) ? (size_t)r.a * N * H + r.c0 : (size_t)r.a * H + r.c0;
    r.ls = (AXIS == AX_Y) ? H : N * H;
    r.cs = 1;
  } else {
    r.isQ = 1;
    r.a = 0;
    r.c0 = (t - MT) * C;
    r.base = (AXIS == AX_Y) ? (size_t)r.c0 * N : (size_t)r.c0;
    r.ls = (AXIS == AX_Y) ? 1 : N;
    r.cs = (AXIS == AX_Y) ? N : 1;
  }
  return r;
}

template <int N, int C, int T>
__device__ __forceinline__ void tile_load(float2* s, const float2* __restrict__ P, const Tile& t) {
  using Lay = ColLayout<C>;
  if (t.cs == 1) {
#pragma unroll 4
    for (int e = threadIdx.x; e < N * (C / 2); e += T) {
      const int i = e / (C / 2), cp = e % (C / 2);
      const float4 v = *reinterpret_cast<const float4*>(P + t.base + (size_t)i * t.ls + 2 * cp);
      s[Lay::phys(i, 2 * cp)] = make_float2(v.x, v.y);
      s[Lay::phys(i, 2 * cp + 1)] = make_float2(v.z, v.w);
    }
  } else {
    for (int e = threadIdx.x; e < N * C; e += T) {
      const int c = e / N, i = e % N;
      s[Lay::phys(i, c)] = P[t.base + (size_t)c * t.cs + (size_t)i * t.ls];
    }
  }
}

template <int N, int C, int T>
__device__ __forceinline__ void tile_store(const float2* s, float2* __restrict__ P, const Tile& t) {
  using Lay = ColLayout<C>;
  if (t.cs == 1) {
    for (int e = threadIdx.x; e < N * (C / 2); e += T) {
      const int i = e / (C / 2), cp = e % (C / 2);
      const float2 v0 = s[Lay::phys(i, 2 * cp)], v1 = s[Lay::phys(i, 2 * cp + 1)];
      *reinterpret_cast<float4*>(P + t.base + (size_t)i * t.ls + 2 * cp) = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
  } else {
    for (int e = threadIdx.x; e < N * C; e += T) {
      const int c = e / N, i = e % N;
      P[t.base + (size_t)c * t.cs + (size_t)i * t.ls] = s[Lay::phys(i, c)];
    }
  }
}

// Stores of the k-space passes along y: the tile of G = iS/k^2 (one slot) goes out twice, scaled by
// kdx into Psi_x and by kdz into Psi_z (kx and kz are constant along a y line; M tiles: kx = t.a,
// kz = column; Nyquist tiles: kx = column, kz = N/2, whose derivative wavenumber is zero).
template <int N, int C, int T>
__device__ __forceinline__ void tile_store_xz(const float2* s, float2* __restrict__ Px, float2* __restrict__ Pz,
                                              const Tile& t, float kf) {
  using Lay = ColLayout<C>;
  constexpr int H = N / 2;
  auto kd = [&](int c, float& kdx, float& kdz) {
    const int ix = t.isQ ? t.c0 + c : t.a, kz = t.isQ ? H : t.c0 + c;
    kdx = (ix == H) ? 0.f : kf * (float)(ix < H ? ix : ix - N);
    kdz = (kz == H) ? 0.f : kf * (float)kz;
  };
  if (t.cs == 1) {
    for (int e = threadIdx.x; e < N * (C / 2); e += T) {
      const int i = e / (C / 2), cp = e % (C / 2);
      const float2 v0 = s[Lay::phys(i, 2 * cp)], v1 = s[Lay::phys(i, 2 * cp + 1)];
      float ax0, az0, ax1, az1;
      kd(2 * cp, ax0, az0);
      kd(2 * cp + 1, ax1, az1);
      const size_t gi = t.base + (size_t)i * t.ls + 2 * cp;
      *reinterpret_cast<float4*>(Px + gi) = make_float4(ax0 * v0.x, ax0 * v0.y, ax1 * v1.x, ax1 * v1.y);
      *reinterpret_cast<float4*>(Pz + gi) = make_float4(az0 * v0.x, az0 * v0.y, az1 * v1.x, az1 * v1.y);
    }
  } else {
    for (int e = threadIdx.x; e < N * C; e += T) {
      const int c = e / N, i = e % N;
      float ax, az;
      kd(c, ax, az);
      const float2 v = s[Lay::phys(i, c)];
      const size_t gi = t.base + (size_t)c * t.cs + (size_t)i * t.ls;
      Px[gi] = cscale(v, ax);
      Pz[gi] = cscale(v, az);
    }
  }
}

// Threads of a strided CTA.  The plain passes move one component per CTA in 16-column (128-byte)
// tiles with 512 threads; the 3-component k-space passes use 4-column (32-byte) tiles with 256
// threads so that three components fit three CTAs per SM.  The k-space passes run along y, whose
// lines are 2 KB strided, so narrow tiles still stream well; the 1 MB-strided x lines get the
// wide tiles.
template <int N, int MODE, int NARROW = 0>
struct SThreads {
  static constexpr bool kK = (MODE == S_DELTA || MODE == S_ITER);
  // 1024-point lines: 128 registers a thread (their butterflies and prefetched values spill at 64),
  // and the k-space passes on 512 threads so that each prefetches 8 values of delta(k) and S
  static constexpr int v = (N >= 1024 && kK) ? 512 : ((!kK && SCols<N, MODE, NARROW>::v == 16) ? 512 : 256);
  static constexpr int minb = N >= 1024 ? (kK ? 1 : 2) : (kK ? 3 : (v == 512 ? 2 : 4));
};

template <int N, int MODE, int NC, int AXIS, int NARROW = 0>
__global__ void __launch_bounds__(SThreads<N, MODE, NARROW>::v, SThreads<N, MODE, NARROW>::minb)
    spass_kernel(const SArgs a) {
  constexpr int T = SThreads<N, MODE, NARROW>::v;
  constexpr int C = SCols<N, MODE, NARROW>::v;
  constexpr int H = N / 2;
  constexpr int NS = (MODE == S_DELTA || MODE == S_ITER) ? 3 : NC;   // smem slots
  using Lay = ColLayout<C>;
  constexpr int TABS = (Plan<N>::kTab + 1) & ~1;
  extern __shared__ float4 ssm[];
  float2* tw = reinterpret_cast<float2*>(ssm);   // stage twiddles of the N-point FFT
  float2* s = tw + TABS;
  __shared__ double red_sh[T / 32];
  const int q0 = blockIdx.y;   // plain passes: the component this CTA transforms
  // k-space passes along y: kx and kz are constant along the line, so the x and z components of
  // k . P travel as A = kdx P_x + kdz P_z (one forward transform for two) and Psi_x, Psi_z leave as
  // kdx G and kdz G of one inverse transform of G = iS/k^2
  constexpr bool RED = (MODE == S_ITER || MODE == S_DELTA) && AXIS == AX_Y;

  if ((MODE == S_FWD || MODE == S_INV) && a.skip_flag && *a.skip_flag != 0) return;   // uniform
  for (int m = threadIdx.x; m < Plan<N>::kTab; m += T) tw[m] = a.tab[m];
  const Tile t = tile_of<N, C, AXIS>(blockIdx.x);

  // ---- load
  if (MODE == S_DELTA) {
    tile_load<N, C, T>(s, t.isQ ? a.dk.Q : a.dk.M, t);
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) tile_load<N, C, T>(s + q * N * C, t.isQ ? a.f[q0 + q].Q : a.f[q0 + q].M, t);
  }
  __syncthreads();

  if (MODE == S_ITER && RED) {
    const float kf = a.g.kf;
    for (int e = threadIdx.x; e < N * C; e += T) {
      const int i = e / C, c = e % C;
      const int ix = t.isQ ? t.c0 + c : t.a, kz = t.isQ ? H : t.c0 + c;
      const float kdx = (ix == H) ? 0.f : kf * (float)(ix < H ? ix : ix - N);
      const float kdz = (kz == H) ? 0.f : kf * (float)kz;
      const int p = Lay::phys(i, c);
      const float2 px = s[p], pz = s[2 * N * C + p];
      s[p] = make_float2(fmaf(kdx, px.x, kdz * pz.x), fmaf(kdx, px.y, kdz * pz.y));
    }
    __syncthreads();
  }

  // ---- S_ITER: fetch delta(k) and the previous source for this thread's elements now, so the
  // loads are in flight during the forward transforms instead of inside the element loop
  constexpr int PE = (N * C + T - 1) / T;
  float2 dkr[MODE == S_ITER ? PE : 1], spr[MODE == S_ITER ? PE : 1];
  if (MODE == S_ITER) {
    const float2* __restrict__ dkp = t.isQ ? a.dk.Q : a.dk.M;
    const float2* __restrict__ spp = t.isQ ? a.sbuf.Q : a.sbuf.M;
#pragma unroll
    for (int k = 0; k < PE; ++k) {
      const int e = threadIdx.x + k * T;
      if ((N * C) % T == 0 || e < N * C) {
        const int i = e / C, c = e % C;
        const size_t gi = t.base + (size_t)i * t.ls + (size_t)c * t.cs;
        dkr[k] = dkp[gi];
        spr[k] = spp[gi];
      }
    }
  }

  // ---- forward transform along the line
  if (MODE == S_FWD || MODE == S_ITER) {
#pragma unroll
    for (int q = 0; q < ((MODE == S_ITER && RED) ? 2 : NC); ++q) Plan<N>::template run<C, T, false, Lay>(s + q * N * C, tw);
  } else if (MODE == S_DELTA) {
    if (!a.d_is_k) Plan<N>::template run<C, T, false, Lay>(s, tw);
  }

  float d2 = 0.f, s2 = 0.f;
  if (MODE == S_DELTA || MODE == S_ITER) {
    const Geometry& g = a.g;
#pragma unroll
    for (int k = 0; k < PE; ++k) {
      const int e = threadIdx.x + k * T;
      if ((N * C) % T != 0 && e >= N * C) break;
      const int i = e / C, c = e % C;
      // wavenumber indices of element (i, c): i runs along the pass axis
      int ix, ky, kz;
      if (AXIS == AX_X) {
        ix = i;
        if (!t.isQ) { ky = t.a; kz = t.c0 + c; } else { ky = t.c0 + c; kz = H; }
      } else {
        ky = i;
        if (!t.isQ) { ix = t.a; kz = t.c0 + c; } else { ix = t.c0 + c; kz = H; }
      }
      const int mx = (ix < H) ? ix : ix - N;
      const int my = (ky < H) ? ky : ky - N;
      const float kx = g.kf * mx, kyf = g.kf * my, kzf = g.kf * kz;
      const float k2 = kx * kx + kyf * kyf + kzf * kzf;
      const int p = Lay::phys(i, c);
      {
        const float kdx = (ix == H) ? 0.f : kx;
        const float kdy = (ky == H) ? 0.f : kyf;
        const float kdz = (kz == H) ? 0.f : kzf;
        const size_t gi = t.base + (size_t)i * t.ls + (size_t)c * t.cs;
        float2* Sp = t.isQ ? a.sbuf.Q : a.sbuf.M;
        float2 S;
        if (MODE == S_DELTA) {
          float2 dk = s[p];
          if (!a.d_is_k) {
            if (a.lognormal && ix == 0 && ky == 0 && kz == 0)
              dk.x -= (float)(a.red[RED_SUM_LOG]);   // subtract N^3 <ln(1+delta)> at k = 0
            (t.isQ ? a.dk.Q : a.dk.M)[gi] = dk;
          }
          S = cscale(dk, a.inv_b);
        } else {
          const float2 dk = dkr[MODE == S_ITER ? k : 0];
          // i k . P
          float dre, dim;
          if (RED) {   // slot 0 holds A = kdx P_x + kdz P_z
            const float2 pa = s[p], py = s[N * C + p];
            dre = fmaf(kdy, py.x, pa.x);
            dim = fmaf(kdy, py.y, pa.y);
          } else {
            const float2 px = s[p], py = s[N * C + p], pz = s[2 * N * C + p];
            dre = kdx * px.x + kdy * py.x + kdz * pz.x;
            dim = kdx * px.y + kdy * py.y + kdz * pz.y;
          }
          S = make_float2(fmaf(a.beta, -dim, dk.x * a.inv_b), fmaf(a.beta, dre, dk.y * a.inv_b));
        }
        if (k2 == 0.f) S = make_float2(0.f, 0.f);
        const float inv_k2 = (k2 > 0.f) ? 1.f / k2 : 0.f;
        if (MODE == S_ITER) {
          const float2 sp = spr[MODE == S_ITER ? k : 0];
          const float wgt = (kz == 0 || kz == H) ? 1.f : 2.f;
          const float fac = wgt * (kdx * kdx + kdy * kdy + kdz * kdz) * inv_k2 * inv_k2;
          const float ddx = S.x - sp.x, ddy = S.y - sp.y;
          d2 = fmaf(fac, ddx * ddx + ddy * ddy, d2);
          s2 = fmaf(fac, S.x * S.x + S.y * S.y, s2);
        }
        Sp[gi] = S;
        // Psi_j = i kd_j S / k^2, with the 1/N^3 of the inverse transform folded in
        const float2 iS = cscale(mul_i(S), inv_k2 * g.inv_n3);
        if (RED) {
          s[p] = iS;                           // G
          s[N * C + p] = cscale(iS, kdy);      // Psi_y
        } else {
          s[p] = cscale(iS, kdx);
          s[N * C + p] = cscale(iS, kdy);
          s[2 * N * C + p] = cscale(iS, kdz);
        }
      }
    }
    __syncthreads();
  }

  // ---- inverse transform along the line
  if (MODE == S_INV || MODE == S_DELTA || MODE == S_ITER) {
#pragma unroll
    for (int q = 0; q < (RED ? 2 : NS); ++q) Plan<N>::template run<C, T, true, Lay>(s + q * N * C, tw);
  }

  // ---- store
  if (RED) {
    tile_store_xz<N, C, T>(s, t.isQ ? a.f[0].Q : a.f[0].M, t.isQ ? a.f[2].Q : a.f[2].M, t, a.g.kf);
    tile_store<N, C, T>(s + N * C, t.isQ ? a.f[1].Q : a.f[1].M, t);
  } else {
#pragma unroll
    for (int q = 0; q < NS; ++q) tile_store<N, C, T>(s + q * N * C, t.isQ ? a.f[q0 + q].Q : a.f[q0 + q].M, t);
  }

  if (MODE == S_ITER) {
    double r0 = block_sum((double)d2, red_sh);
    double r1 = block_sum((double)s2, red_sh);
    if (threadIdx.x == 0) {
      a.partials[2 * blockIdx.x + 0] = r0;
      a.partials[2 * blockIdx.x + 1] = r1;
    }
  }
}

template <int N, int MODE, int NARROW = 0>
constexpr size_t spass_smem(int nslots) {
  return sizeof(float2) * ((size_t)((Plan<N>::kTab + 1) & ~1) + (size_t)nslots * N * SCols<N, MODE, NARROW>::v);
}

// ------------------------------------------------------------------------------------------------
// The k-space update along y for N = 512 = 8 x 8 x 8.  With three radix-8 Stockham stages the
// butterfly j of the last forward stage produces X[j + 64 r] (r = 0..7), and these are exactly the
// inputs of butterfly j of the first inverse stage.  So each thread loads its 8 points of a column
// straight from global memory into the first forward stage, keeps the last forward stage's outputs
// in registers for the source update, starts the inverse transform on them, and stores the last
// inverse stage straight to global memory: two shared-memory round trips per transform instead of
// three plus the staging of loads, stores and the update.  The arithmetic of every butterfly is the
// same as in the generic stages.
// ------------------------------------------------------------------------------------------------
template <int N, int C>
struct KIter8 {
  static_assert(N == 512, "three radix-8 stages");
  static constexpr int T = (N / 8) * C;        // one butterfly of one column per thread and stage
  static constexpr int kMinBlocks = T <= 256 ? 2 : 1;
  static constexpr int TAB = (Plan<N>::kTab + 1) & ~1;
  // one buffer per transformed line: the x and z terms share one (see kiter8_kernel)
  static constexpr size_t smem = sizeof(float2) * ((size_t)TAB + 2 * (size_t)N * C);
};

// The 512-point transforms of K lines of one column (K = 2 in the update: A and P_y forward, G and
// Psi_y inverse; K = 1 for delta), stage by stage together (one buffer each, so a stage needs one
// barrier for all K): v[q][r] = x_q[j + 64 r] in, X_q[j + 64 r] out.
template <bool INV, int N, int C, int K>
__device__ __forceinline__ void r512_lines(float2 (&v)[K][8], float2* __restrict__ s, const float2* __restrict__ tw,
                                            int j, int col) {
  using Lay = ColLayout<C>;
  constexpr int B = N * C;
#pragma unroll
  for (int q = 0; q < K; ++q) {                          // stage 1 (NS = 1): no twiddles
    Dft<8, INV>::run(v[q]);
#pragma unroll
    for (int r = 0; r < 8; ++r) s[q * B + Lay::phys(8 * j + r, col)] = v[q][r];
  }
  __syncthreads();
  const int k = j & 7;
#pragma unroll
  for (int q = 0; q < K; ++q) {                          // stage 2 (NS = 8)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[q][r] = s[q * B + Lay::phys(j + 64 * r, col)];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      float2 w = tw[(r - 1) * 8 + k];
      if (INV) w.y = -w.y;
      v[q][r] = cmul(v[q][r], w);
    }
    Dft<8, INV>::run(v[q]);
  }
  __syncthreads();
  const int base = (j >> 3) * 64 + k;
#pragma unroll
  for (int q = 0; q < K; ++q)
#pragma unroll
    for (int r = 0; r < 8; ++r) s[q * B + Lay::phys(base + 8 * r, col)] = v[q][r];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {                          // stage 3 (NS = 64)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[q][r] = s[q * B + Lay::phys(j + 64 * r, col)];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      float2 w = tw[56 + (r - 1) * 64 + j];
      if (INV) w.y = -w.y;
      v[q][r] = cmul(v[q][r], w);
    }
    Dft<8, INV>::run(v[q]);
  }
  __syncthreads();                                       // the buffers are reused
}

// The start's k-space pass along y for N = 512 (S_DELTA): the y transform of delta (unless delta(k)
// is already stored), delta(k) and S_-1 = delta/b stored, Z[delta/b] with two inverse y transforms
// (G and Psi_y, as the update kernel leaves them), the first and last stages in registers.
template <int N, int C>
__global__ void __launch_bounds__(KIter8<N, C>::T, KIter8<N, C>::kMinBlocks) kdelta8_kernel(const SArgs a) {
  constexpr int T = KIter8<N, C>::T;
  constexpr int H = N / 2;
  extern __shared__ float4 ssm[];
  float2* tw = reinterpret_cast<float2*>(ssm);
  float2* s = tw + KIter8<N, C>::TAB;
  for (int m = threadIdx.x; m < Plan<N>::kTab; m += T) tw[m] = a.tab[m];
  const Tile t = tile_of<N, C, AX_Y>(blockIdx.x);
  const int col = threadIdx.x % C, j = threadIdx.x / C;
  float2* __restrict__ dkp = t.isQ ? a.dk.Q : a.dk.M;
  float2 d[1][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) d[0][r] = dkp[t.base + (size_t)(j + 64 * r) * t.ls + (size_t)col * t.cs];
  __syncthreads();   // twiddles
  if (!a.d_is_k) r512_lines<false, N, C, 1>(d, s, tw, j, col);

  const Geometry& g = a.g;
  float2* Sp = t.isQ ? a.sbuf.Q : a.sbuf.M;
  float2 v[2][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int ky = j + 64 * r;
    int ix, kz;
    if (!t.isQ) { ix = t.a; kz = t.c0 + col; } else { ix = t.c0 + col; kz = H; }
    const int mx = (ix < H) ? ix : ix - N;
    const int my = (ky < H) ? ky : ky - N;
    const float kx = g.kf * mx, kyf = g.kf * my, kzf = g.kf * kz;
    const float k2 = kx * kx + kyf * kyf + kzf * kzf;
    const float kdy = (ky == H) ? 0.f : kyf;
    const size_t gi = t.base + (size_t)ky * t.ls + (size_t)col * t.cs;
    float2 dk = d[0][r];
    if (!a.d_is_k) {
      if (a.lognormal && ix == 0 && ky == 0 && kz == 0) dk.x -= (float)(a.red[RED_SUM_LOG]);   // N^3 <ln(1+delta)>
      dkp[gi] = dk;
    }
    float2 S = cscale(dk, a.inv_b);
    if (k2 == 0.f) S = make_float2(0.f, 0.f);
    const float inv_k2 = (k2 > 0.f) ? 1.f / k2 : 0.f;
    Sp[gi] = S;
    const float2 iS = cscale(mul_i(S), inv_k2 * g.inv_n3);
    v[0][r] = iS;
    v[1][r] = cscale(iS, kdy);
  }
  r512_lines<true, N, C, 2>(v, s, tw, j, col);
  {
    // G (Psi_x = kdx G, Psi_z = kdz G) in the third field, Psi_y in the second, as the update
    // kernel leaves them
    float2* __restrict__ dy = t.isQ ? a.f[1].Q : a.f[1].M;
    float2* __restrict__ dg = t.isQ ? a.f[2].Q : a.f[2].M;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const size_t gi = t.base + (size_t)(j + 64 * r) * t.ls + (size_t)col * t.cs;
      dy[gi] = v[1][r];
      dg[gi] = v[0][r];
    }
  }
}

// The line transform along x for N = 512: the first radix-8 stage reads its inputs straight from
// global memory and the last writes its outputs straight back, so shared memory carries only the
// middle stage (the generic pass also stages the loads and stores).  Tiles of C adjacent columns,
// 64 butterflies per column and stage, NB per thread.
template <int C>
struct XLine8 {
  static constexpr int T = 512;
  static constexpr int NB = 64 * C / T;        // butterflies per thread and stage
  static constexpr int TAB = (Plan<512>::kTab + 1) & ~1;
  static constexpr size_t smem = sizeof(float2) * ((size_t)TAB + (size_t)512 * C);
};

// The three radix-8 stages of a 512-point transform over C columns, the thread's NB butterflies
// (j_b = jb + b T / C) with the first stage's inputs and the last stage's outputs handled one
// butterfly at a time: ld(b, x) supplies x[r] = X[j_b + 64 r] and st(b, y) takes the outputs
// y[r] = Y[j_b + 64 r], so only the middle stage holds all NB butterflies in registers (it reads
// and writes shared memory in place).  Starts by writing s: a caller that ran it before syncs first.
template <bool INV, int C, class Ld, class St>
__device__ __forceinline__ void xline8_io(float2* __restrict__ s, const float2* __restrict__ tw, int jb, int col,
                                          Ld&& ld, St&& st) {
  constexpr int T = XLine8<C>::T, NB = XLine8<C>::NB;
  using Lay = ColLayout<C>;
#pragma unroll
  for (int b = 0; b < NB; ++b) {                          // stage 1 (NS = 1)
    const int j = jb + b * (T / C);
    float2 x[8];
    ld(b, x);
    Dft<8, INV>::run(x);
#pragma unroll
    for (int r = 0; r < 8; ++r) s[Lay::phys(8 * j + r, col)] = x[r];
  }
  __syncthreads();
  float2 v[NB][8];
#pragma unroll
  for (int b = 0; b < NB; ++b) {                          // stage 2 (NS = 8)
    const int j = jb + b * (T / C), k = j & 7;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[b][r] = s[Lay::phys(j + 64 * r, col)];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      float2 w = tw[(r - 1) * 8 + k];
      if (INV) w.y = -w.y;
      v[b][r] = cmul(v[b][r], w);
    }
    Dft<8, INV>::run(v[b]);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = jb + b * (T / C), base = (j >> 3) * 64 + (j & 7);
#pragma unroll
    for (int r = 0; r < 8; ++r) s[Lay::phys(base + 8 * r, col)] = v[b][r];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {                          // stage 3 (NS = 64)
    const int j = jb + b * (T / C);
    float2 y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) y[r] = s[Lay::phys(j + 64 * r, col)];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      float2 w = tw[56 + (r - 1) * 64 + j];
      if (INV) w.y = -w.y;
      y[r] = cmul(y[r], w);
    }
    Dft<8, INV>::run(y);
    st(b, y);
  }
}

// PAIR = false: one component per CTA (blockIdx.y).  PAIR = true: the vector passes between the
// register-fused k-space pass (y) and the fused z pass, which carry vectors in reduced forms: kx and
// kz (kdx, kdz: zero at the Nyquist index) are constant along a y line, so the y pass needs
// A = kdx P_x + kdz P_z and P_y and returns G (Psi_x = kdx G, Psi_z = kdz G) and Psi_y; and the
// observer offset dy (a fixed line of sight's y component) is constant along an x line, so the z
// pass hands over psi^ = r2c_z(psi) and Z^ = r2c_z(dz psi) with P_x = dx psi^, P_y = dy psi^.
// Two CTAs per tile, on adjacent block indices (role = blockIdx.x & 1), so that a field both read
// comes from HBM once and from the L2 the second time:
//   inverse: role 1 transforms Psi_y in the second field in place; role 0 transforms G (third field)
//            twice, Psi_x = IFFT_x(kdx G) into the first and Psi_z = kdz IFFT_x(G) into the third;
//   inverse in C form (a.cform, while the loop runs): the projection pass needs only
//            C = dx Psi_x + dy Psi_y and Psi_z, and dx varies along the x line (the output index)
//            while dy is the tile's constant, so role 0 leaves C = dx IFFT_x(kdx G) + dy IFFT_x(Psi_y)
//            in the first field and role 1 Psi_z = kdz IFFT_x(G) in the fourth (wf): two fields
//            written instead of three, and the projection pass reads two;
//   forward: role 1 leaves P_y = dy FFT_x(psi^) (first field) in the second; role 0 leaves
//            A = kdx FFT_x(dx psi^) + kdz FFT_x(Z^) in the third (its first product goes through the
//            L2 and is read back by the thread that wrote it).
__device__ __forceinline__ uint32_t opaque_u32(uint32_t x) {
  asm volatile("" : "+r"(x));
  return x;
}

template <bool INV, int C, bool PAIR>
__global__ void __launch_bounds__(XLine8<C>::T, 2) xline8_kernel(const SArgs a) {
  constexpr int N = 512, H = N / 2, T = XLine8<C>::T, NB = XLine8<C>::NB;
  extern __shared__ float4 ssm[];
  float2* tw = reinterpret_cast<float2*>(ssm);
  float2* s = tw + XLine8<C>::TAB;
  if (!INV && a.skip_flag && *a.skip_flag != 0) return;   // uniform: device loop already converged
  for (int m = threadIdx.x; m < Plan<N>::kTab; m += T) tw[m] = a.tab[m];
  const int role = PAIR ? (int)(blockIdx.x & 1) : (int)blockIdx.y;
  // tiles of every y-plane, or of the planes [ybeg, ybeg + ycount): their M tiles (ky, kz block)
  // and the Nyquist tiles that hold their ky columns
  int ti = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  if (a.ycount) {
    const int mt = a.ycount * (H / C);
    ti = ti < mt ? a.ybeg * (H / C) + ti : N * (H / C) + a.ybeg / C + (ti - mt);
  }
  const Tile t = tile_of<N, C, AX_X>(ti);
  const int col = threadIdx.x % C, jb = threadIdx.x / C;
  // element offsets fit 32 bits (at most N^3 / 2 complex points per field)
  const uint32_t o0 = (uint32_t)t.base + (uint32_t)(col * t.cs) + (uint32_t)jb * (uint32_t)t.ls;
  const uint32_t ls = (uint32_t)t.ls;
  // element offset of point (b, r) of this thread; every load and store re-derives the base through
  // an opaque copy, so no offset is kept live across a transform
  auto off = [&](uint32_t base, int b, int r) { return base + (uint32_t)(b * (T / C) + 64 * r) * ls; };
  auto load = [&](const float2* __restrict__ P) {
    return [=, &off](int b, float2 (&x)[8]) {
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = P[off(o0, b, r)];
    };
  };
  auto store = [&](float2* __restrict__ P, float scale) {
    return [=, &off](int b, const float2 (&y)[8]) {
      const uint32_t o = opaque_u32(o0);
#pragma unroll
      for (int r = 0; r < 8; ++r) P[off(o, b, r)] = cscale(y[r], scale);
    };
  };
  const Geometry& g = a.g;
  const bool cf = PAIR && INV && a.cform && !(a.loop_flag && *a.loop_flag == 1);
  if (!PAIR || (INV && role == 1 && !cf)) {
    float2* __restrict__ P = t.isQ ? a.f[role].Q : a.f[role].M;
    xline8_io<INV, C>(s, tw, jb, col, load(P), store(P, 1.f));
    return;
  }
  float2* __restrict__ P0 = t.isQ ? a.f[0].Q : a.f[0].M;
  float2* __restrict__ P1 = t.isQ ? a.f[1].Q : a.f[1].M;
  float2* __restrict__ P2 = t.isQ ? a.f[2].Q : a.f[2].M;
  const float dy = g.los_mode == 1 ? g.los.y : g.off[N + (t.isQ ? t.c0 + col : t.a)];
  if (!INV && role == 1) {   // P_y = dy FFT_x(psi^)
    xline8_io<INV, C>(s, tw, jb, col, load(P0), store(P1, dy));
    return;
  }
  const float kf = g.kf;
  const float kdz = t.isQ ? 0.f : kf * (float)(t.c0 + col);   // M tiles: kz < N/2; Q tiles: kz = N/2
  // the line index i is kx in Fourier space and x in configuration space
  auto kdx = [&](int b, int r) {
    const int i = jb + b * (T / C) + 64 * r;
    return i == H ? 0.f : kf * (float)(i < H ? i : i - N);
  };
  auto dxv = [&](int b, int r) { return g.los_mode == 1 ? g.los.x : g.off[jb + b * (T / C) + 64 * r]; };
  // loads of G scaled by kdx (the inverse's x component)
  auto load_kdx_g = [&](int b, float2 (&x)[8]) {
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = cscale(P2[off(o0, b, r)], kdx(b, r));
  };
  if (cf) {
    // both roles start on G, so the pair reads it from HBM once
    if (role == 1) {   // Psi_z = kdz IFFT_x(G)
      float2* __restrict__ W = t.isQ ? a.wf.Q : a.wf.M;
      xline8_io<INV, C>(s, tw, jb, col, load(P2), store(W, kdz));
      return;
    }
    // role 0: Psi_x = IFFT_x(kdx G) parked in the first field, then C = fmaf(dx, Psi_x, dy Psi_y),
    // rounded exactly as the projection pass forms it from the three components
    xline8_io<INV, C>(s, tw, jb, col, load_kdx_g, store(P0, 1.f));
    __syncthreads();   // s is rewritten by the second transform
    xline8_io<INV, C>(s, tw, jb, col, load(P1), [&](int b, const float2 (&y)[8]) {   // IFFT_x(Psi_y)
      const uint32_t o = opaque_u32(o0);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 x = P0[off(o, b, r)];   // this thread's own Psi_x
        const float d = dxv(b, r);
        P0[off(o, b, r)] = make_float2(fmaf(d, x.x, dy * y[r].x), fmaf(d, x.y, dy * y[r].y));
      }
    });
    return;
  }
  if (INV) {   // three components: Psi_x = IFFT_x(kdx G) into the first field, Psi_z = kdz IFFT_x(G)
    xline8_io<INV, C>(s, tw, jb, col, load_kdx_g, store(P0, 1.f));
    __syncthreads();   // s is rewritten by the second transform
    xline8_io<INV, C>(s, tw, jb, col, load(P2), store(P2, kdz));
    return;
  }
  // forward: kdz FFT_x(Z^) into the third field, then A = kdx FFT_x(dx psi^) + that
  xline8_io<INV, C>(s, tw, jb, col, load(P2), store(P2, kdz));
  __syncthreads();   // s is rewritten by the second transform
  xline8_io<INV, C>(s, tw, jb, col,
                    [&](int b, float2 (&x)[8]) {
#pragma unroll
                      for (int r = 0; r < 8; ++r) x[r] = cscale(P0[off(o0, b, r)], dxv(b, r));
                    },
                    [&](int b, const float2 (&y)[8]) {   // FFT_x(dx psi^)
                      const uint32_t o = opaque_u32(o0);
#pragma unroll
                      for (int r = 0; r < 8; ++r) {
                        const float2 x = P2[off(o, b, r)];   // this thread's own kdz FFT_x(Z^)
                        const float k = kdx(b, r);
                        P2[off(o, b, r)] = make_float2(fmaf(k, y[r].x, x.x), fmaf(k, y[r].y, x.y));
                      }
                    });
}

// One tile of the source update (Eq. iterative) from registers: v[0] = A and v[1] = P_y along the y
// line (Fourier x and z, configuration y), dk = delta(k) and sp = S_(n-1) at the thread's 8 points
// (already in Fourier y).  Forward y FFT, S_n = delta/b + beta i k . P_n, the Parseval norms
// (accumulated into d2, s2), Psi_n+1 = i kd S_n / k^2 as G (third field) and Psi_y (second field),
// inverse y FFT, stores.  kx and kz are constant along the y line, so the x and z terms of k . P
// arrive combined, A = kdx P_x + kdz P_z (the forward x pass forms it; FFT_y is linear), and
// Psi_x, Psi_z leave as one field G with Psi_x = kdx G, Psi_z = kdz G (the inverse x pass separates
// them).  s is written first: a caller that used it before syncs first.
template <int N, int C>
__device__ __forceinline__ void kiter_tile(const SArgs& a, const Tile& t, float2 (&v)[2][8], const float2 (&dk)[8],
                                           const float2 (&sp)[8], float2* __restrict__ s,
                                           const float2* __restrict__ tw, int j, int col, float& d2, float& s2) {
  constexpr int H = N / 2;
  const Geometry& g = a.g;
  int ix, kz;
  if (!t.isQ) { ix = t.a; kz = t.c0 + col; } else { ix = t.c0 + col; kz = H; }
  const int mx = (ix < H) ? ix : ix - N;
  const float kx = g.kf * mx, kzf = g.kf * kz;
  const float kdx = (ix == H) ? 0.f : kx;
  const float kdz = (kz == H) ? 0.f : kzf;
  r512_lines<false, N, C, 2>(v, s, tw, j, col);
  float2* Sp = t.isQ ? a.sbuf.Q : a.sbuf.M;
  const float kxz2 = kx * kx + kzf * kzf, kdxz2 = kdx * kdx + kdz * kdz;
  const float wgt = (kz == 0 || kz == H) ? 1.f : 2.f;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int ky = j + 64 * r;
    const int my = (ky < H) ? ky : ky - N;
    const float kyf = g.kf * my;
    const float k2 = kxz2 + kyf * kyf;
    const float kdy = (ky == H) ? 0.f : kyf;
    const float2 pa = v[0][r], py = v[1][r];
    const float dre = fmaf(kdy, py.x, pa.x);
    const float dim = fmaf(kdy, py.y, pa.y);
    float2 S = make_float2(fmaf(a.beta, -dim, dk[r].x * a.inv_b), fmaf(a.beta, dre, dk[r].y * a.inv_b));
    if (k2 == 0.f) S = make_float2(0.f, 0.f);
    const float inv_k2 = (k2 > 0.f) ? 1.f / k2 : 0.f;
    const float fac = wgt * (kdxz2 + kdy * kdy) * inv_k2 * inv_k2;
    const float ddx = S.x - sp[r].x, ddy = S.y - sp[r].y;
    d2 = fmaf(fac, ddx * ddx + ddy * ddy, d2);
    s2 = fmaf(fac, S.x * S.x + S.y * S.y, s2);
    Sp[t.base + (size_t)ky * t.ls + (size_t)col * t.cs] = S;
    const float2 iS = cscale(mul_i(S), inv_k2 * g.inv_n3);
    v[0][r] = iS;
    v[1][r] = cscale(iS, kdy);
  }
  r512_lines<true, N, C, 2>(v, s, tw, j, col);
  float2* __restrict__ dy = t.isQ ? a.f[1].Q : a.f[1].M;
  float2* __restrict__ dg = t.isQ ? a.f[2].Q : a.f[2].M;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const size_t gi = t.base + (size_t)(j + 64 * r) * t.ls + (size_t)col * t.cs;
    dy[gi] = v[1][r];
    dg[gi] = v[0][r];
  }
}

// The tile's four inputs straight from global memory: A (third field), P_y (second), delta(k), S.
template <int N, int C>
__device__ __forceinline__ void kiter_load(const SArgs& a, const Tile& t, int j, int col, float2 (&v)[2][8],
                                           float2 (&dk)[8], float2 (&sp)[8]) {
  const float2* __restrict__ dkp = t.isQ ? a.dk.Q : a.dk.M;
  const float2* __restrict__ spp = t.isQ ? a.sbuf.Q : a.sbuf.M;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const size_t gi = t.base + (size_t)(j + 64 * r) * t.ls + (size_t)col * t.cs;
    v[0][r] = (t.isQ ? a.f[2].Q : a.f[2].M)[gi];
    v[1][r] = (t.isQ ? a.f[1].Q : a.f[1].M)[gi];
    dk[r] = dkp[gi];
    sp[r] = spp[gi];
  }
}

template <int N, int C>
__global__ void __launch_bounds__(KIter8<N, C>::T, KIter8<N, C>::kMinBlocks) kiter8_kernel(const SArgs a) {
  constexpr int T = KIter8<N, C>::T;
  extern __shared__ float4 ssm[];
  float2* tw = reinterpret_cast<float2*>(ssm);
  float2* s = tw + KIter8<N, C>::TAB;
  __shared__ double red_sh[T / 32];
  for (int m = threadIdx.x; m < Plan<N>::kTab; m += T) tw[m] = a.tab[m];
  const Tile t = tile_of<N, C, AX_Y>(blockIdx.x);
  const int col = threadIdx.x % C, j = threadIdx.x / C;
  // every global read of the tile up front
  float2 v[2][8], dk[8], sp[8];
  kiter_load<N, C>(a, t, j, col, v, dk, sp);
  __syncthreads();   // twiddles
  float d2 = 0.f, s2 = 0.f;
  kiter_tile<N, C>(a, t, v, dk, sp, s, tw, j, col, d2, s2);
  double r0 = block_sum((double)d2, red_sh);
  double r1 = block_sum((double)s2, red_sh);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x + 0] = r0;
    a.partials[2 * blockIdx.x + 1] = r1;
  }
}

// ---- the source update with its inputs streamed by the tensor memory accelerator ---------------
// Persistent CTAs (two per SM) walk the Fourier-x/z tiles; a tile's four inputs (A, P_y, delta(k),
// S_(n-1): four [512 y][4 kz] float2 boxes of a 3-D map over the half grid M [kx][ky][kz < N/2]) land
// in one shared-memory stage by cp.async.bulk.tensor, completing on an mbarrier.  As soon as the
// threads have copied the tile into their registers the next tile's copies are issued into the same
// stage, so they stream in while this tile's transforms and stores run.  The Nyquist tiles (a
// different layout, 1/257 of the data) follow with plain loads.  Each CTA's norms go to its
// partials; the rest of the regular grid's partials are zeroed so the reduction over them is
// unchanged.  Every wait is bounded: a wait that gives up writes NaN norms (the device loop then
// stops with RECON_ERR_NONFINITE) and the CTA returns.
template <int N, int C>
struct KTma {
  static constexpr int T = KIter8<N, C>::T;
  static constexpr size_t kS = sizeof(float2) * ((size_t)KIter8<N, C>::TAB + 2 * (size_t)N * C);
  static constexpr size_t kBufOff = (kS + 127) & ~(size_t)127;
  static constexpr size_t kField = sizeof(float2) * (size_t)N * C;   // one field's tile
  static constexpr size_t kBarOff = kBufOff + 4 * kField;
  static constexpr size_t smem = kBarOff + 16;
  static constexpr uint32_t kTx = 4u * (uint32_t)kField;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

template <int N, int C>
__global__ void __launch_bounds__(KIter8<N, C>::T, 2) kiter8_tma_kernel(const SArgs a,
                                                                       const __grid_constant__ KIterMaps maps) {
  using K = KTma<N, C>;
  constexpr int T = K::T, H = N / 2, MT = N * (H / C), QT = N / C;
  constexpr int kGridPartials = MT + QT;   // the regular grid whose partials the reduction reads
  extern __shared__ __align__(128) float4 ssm[];
  float2* tw = reinterpret_cast<float2*>(ssm);
  float2* s = tw + KIter8<N, C>::TAB;
  const float2* buf = reinterpret_cast<const float2*>(reinterpret_cast<char*>(ssm) + K::kBufOff);
  uint64_t* bar_p = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ssm) + K::kBarOff);
  __shared__ double red_sh[T / 32];
  __shared__ int give_up;
  const uint32_t bar = smem_addr(bar_p), dst = smem_addr(buf);
  for (int m = threadIdx.x; m < Plan<N>::kTab; m += T) tw[m] = a.tab[m];
  if (threadIdx.x == 0) {
    give_up = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  const int col = threadIdx.x % C, j = threadIdx.x / C;
  auto issue = [&](int tt) {   // thread 0: the four fields' boxes of tile tt
    const int kx = tt / (H / C), c0 = (tt % (H / C)) * C;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(K::kTx) : "memory");
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        tma_load3(dst + (uint32_t)(q * K::kField + h * (K::kField / 2)), &maps.m[q], c0, 256 * h, kx, bar);
  };
  float d2 = 0.f, s2 = 0.f;
  float2 v[2][8], dk[8], sp[8];
  uint32_t parity = 0;
  if (threadIdx.x == 0 && (int)blockIdx.x < MT) issue(blockIdx.x);
  for (int tt = blockIdx.x; tt < MT; tt += gridDim.x) {
    // bounded wait for the tile's copies: two seconds of the global timer at most
    bool ok = bar_try_wait(bar, parity);
    if (!ok) {
      unsigned long long t0;
      asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
      for (;;) {
        if ((ok = bar_try_wait(bar, parity))) break;
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t1));
        if (t1 - t0 > 2000000000ull) break;
      }
    }
    if (!ok) give_up = 1;
    __syncthreads();
    if (give_up) break;
    parity ^= 1u;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (j + 64 * r) * C + col;
      v[0][r] = buf[e];
      v[1][r] = buf[N * C + e];
      dk[r] = buf[2 * N * C + e];
      sp[r] = buf[3 * N * C + e];
    }
    __syncthreads();   // the stage is free (and s may be rewritten)
    if (threadIdx.x == 0 && tt + (int)gridDim.x < MT) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(tt + gridDim.x);
    }
    kiter_tile<N, C>(a, tile_of<N, C, AX_Y>(tt), v, dk, sp, s, tw, j, col, d2, s2);
  }
  if (!give_up) {
    for (int q = blockIdx.x; q < QT; q += gridDim.x) {   // Nyquist tiles: plain loads
      const Tile t = tile_of<N, C, AX_Y>(MT + q);
      kiter_load<N, C>(a, t, j, col, v, dk, sp);
      __syncthreads();   // s may be rewritten
      kiter_tile<N, C>(a, t, v, dk, sp, s, tw, j, col, d2, s2);
    }
  }
  double r0 = block_sum((double)d2, red_sh);
  double r1 = block_sum((double)s2, red_sh);
  if (threadIdx.x == 0) {
    if (give_up) r0 = r1 = __longlong_as_double(0x7ff8000000000000ll);   // NaN: the loop stops
    a.partials[2 * blockIdx.x + 0] = r0;
    a.partials[2 * blockIdx.x + 1] = r1;
  }
  for (int b = blockIdx.x + gridDim.x + threadIdx.x * gridDim.x; b < kGridPartials; b += T * gridDim.x) {
    a.partials[2 * b + 0] = 0.0;
    a.partials[2 * b + 1] = 0.0;
  }
}

// Stage twiddle tables of the N-point (strided passes) and N/2-point (Z pass) plans, built once
// from the float32 table of exp(-2 pi i m / N) that the host computed in float64.
template <int N>
__global__ void build_tables_kernel(const float2* __restrict__ tw, float2* tabS, float2* tabZ) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  Plan<N>::template fill<1>(tabS, tw, tid, nthr);
  Plan<N / 2>::template fill<2>(tabZ, tw, tid, nthr);
}

// ------------------------------------------------------------------------------------------------
// Launch tables
// ------------------------------------------------------------------------------------------------
template <class K>
static cudaError_t launch_with_smem(K kern, int blocks, int threads, size_t smem, cudaStream_t st, const void* arg) {
  static_assert(sizeof(K) > 0, "");
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<void*>(arg)};
  return cudaLaunchKernel((const void*)kern, dim3(blocks), dim3(threads), args, smem, st);
}

template <int N>
struct MeshImpl {
  static constexpr int kZBlocks = N * N / kZWarps;   // rows / warps per CTA: upper bound of the Z grid
  template <int M_, int NARROW = 0>
  static constexpr int sblocks() {
    return N * ((N / 2) / SCols<N, M_, NARROW>::v) + N / SCols<N, M_, NARROW>::v;
  }
  static constexpr int kSBlocks = sblocks<S_ITER>();   // grid of the k-space pass (its partials)

  // persistent Z launch: exactly as many CTAs as fit on the device at once (occupancy x SMs),
  // never more than one row per warp
  template <int M_, int NC_>
  static cudaError_t zlaunch(const ZArgs& a, cudaStream_t st, int* grid_out) {
    static int grid = 0;
    const size_t smem = zpass_smem<N, NC_>(M_);
    const void* k = (const void*)zpass_kernel<N, M_, NC_>;
    if (grid == 0) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int dev = 0, sm = 0, occ = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kZThreads, smem)) != cudaSuccess) return e;
      if (occ < 1) return cudaErrorInvalidConfiguration;
      grid = occ * sm < kZBlocks ? occ * sm : kZBlocks;
    }
    if (grid_out) *grid_out = grid;
    void* args[] = {const_cast<ZArgs*>(&a)};
    return cudaLaunchKernel(k, dim3(grid), dim3(kZThreads), args, smem, st);
  }

  template <int M_>
  static cudaError_t zfused(const ZArgs& a, cudaStream_t st, int* grid_out) {
    if constexpr (N == 512) {
      static int grid = 0;
      const void* k = (const void*)zfused8_kernel<N, M_>;
      const size_t smem = ZProj8<N>::smem;
      if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sm = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kZThreads, smem)) != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        grid = occ * sm < kZBlocks ? occ * sm : kZBlocks;
      }
      if (a.ycount && (a.ybeg < 0 || a.ycount < 0 || a.ybeg + a.ycount > N)) return cudaErrorInvalidValue;
      const int rows_blocks = a.ycount ? (N * a.ycount + kZWarps - 1) / kZWarps : kZBlocks;
      const int g = grid < rows_blocks ? grid : rows_blocks;
      if (grid_out) *grid_out = g;
      void* args[] = {const_cast<ZArgs*>(&a)};
      return cudaLaunchKernel(k, dim3(g), dim3(kZThreads), args, smem, st);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t zdelta_fused(const ZArgs& a, cudaStream_t st, int* grid_out) {
    if constexpr (N == 512) {
      static int grid = 0;
      const void* k = (const void*)zdelta8_kernel<N>;
      const size_t smem = ZDelta8<N>::smem;
      if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sm = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kZThreads, smem)) != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        grid = occ * sm < kZBlocks ? occ * sm : kZBlocks;
      }
      if (grid_out) *grid_out = grid;
      void* args[] = {const_cast<ZArgs*>(&a)};
      return cudaLaunchKernel(k, dim3(grid), dim3(kZThreads), args, smem, st);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t zpass(int mode, int nc, const ZArgs& a, cudaStream_t st, int* grid_out) {
    if constexpr (N == 512) {
      if (mode == Z_DELTA && nc == 2 && !a.generic && a.ntap <= ZDelta8<N>::KT) return zdelta_fused(a, st, grid_out);
      if (nc == 3 && !a.generic) {
        if (mode == Z_PROJ) return zfused<Z_PROJ>(a, st, grid_out);
        if (mode == Z_RADIAL) return zfused<Z_RADIAL>(a, st, grid_out);
        if (mode == Z_WARM && a.clevel >= 1) return zfused<Z_WARM>(a, st, grid_out);
        if (mode == Z_USTART) return zfused<Z_USTART>(a, st, grid_out);
      }
    }
#define RG_Z(M_, NC_) \
  if (mode == M_ && nc == NC_) return zlaunch<M_, NC_>(a, st, grid_out);
    RG_Z(Z_FWD, 1) RG_Z(Z_INV, 1) RG_Z(Z_DELTA, 2) RG_Z(Z_PROJ, 3) RG_Z(Z_FINAL, 3) RG_Z(Z_USTART, 3)
    RG_Z(Z_RADIAL, 3) RG_Z(Z_WARM, 3)
#undef RG_Z
    return cudaErrorInvalidValue;
  }

  template <int M_, int NC_, int AX_, int NARROW = 0>
  static cudaError_t slaunch(const SArgs& a, cudaStream_t st, int ncomp) {
    const size_t smem = spass_smem<N, M_, NARROW>((M_ == S_DELTA || M_ == S_ITER) ? 3 : NC_);
    const void* k = (const void*)spass_kernel<N, M_, NC_, AX_, NARROW>;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    void* args[] = {const_cast<SArgs*>(&a)};
    return cudaLaunchKernel(k, dim3(sblocks<M_, NARROW>(), ncomp), dim3(SThreads<N, M_, NARROW>::v), args, smem,
                            st);
  }

  static cudaError_t klaunch(const SArgs& a, cudaStream_t st) {
    if constexpr (N == 512) {
      constexpr int C = SCols<N, S_ITER>::v;
      if (a.tmaps) {   // inputs streamed by TMA into persistent CTAs, two per SM
        const void* k = (const void*)kiter8_tma_kernel<N, C>;
        static int grid = 0;
        if (grid == 0) {
          cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KTma<N, C>::smem);
          if (e != cudaSuccess) return e;
          int dev = 0, sm = 0, occ = 0;
          if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
          if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
          if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, KTma<N, C>::T, KTma<N, C>::smem)) != cudaSuccess)
            return e;
          if (occ < 1) return cudaErrorInvalidConfiguration;
          grid = occ * sm;
        }
        void* args[] = {const_cast<SArgs*>(&a), const_cast<KIterMaps*>(a.tmaps)};
        return cudaLaunchKernel(k, dim3(grid), dim3(KTma<N, C>::T), args, KTma<N, C>::smem, st);
      }
      const void* k = (const void*)kiter8_kernel<N, C>;
      static bool attr = false;
      if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KIter8<N, C>::smem);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      void* args[] = {const_cast<SArgs*>(&a)};
      return cudaLaunchKernel(k, dim3(sblocks<S_ITER>()), dim3(KIter8<N, C>::T), args, KIter8<N, C>::smem, st);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t dlaunch(const SArgs& a, cudaStream_t st) {
    if constexpr (N == 512) {
      constexpr int C = SCols<N, S_DELTA>::v;
      const void* k = (const void*)kdelta8_kernel<N, C>;
      static bool attr = false;
      if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KIter8<N, C>::smem);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      void* args[] = {const_cast<SArgs*>(&a)};
      return cudaLaunchKernel(k, dim3(sblocks<S_DELTA>()), dim3(KIter8<N, C>::T), args, KIter8<N, C>::smem, st);
    }
    return cudaErrorInvalidValue;
  }

  // x lines for N = 512: C = 16 (128-byte rows) or 8 columns (line tile option); pair: the vector
  // passes of the register-fused k-space path (two CTA kinds along gridDim.y, see xline8_kernel)
  template <int C, bool PAIR>
  static cudaError_t xlaunch_c(bool inv, const SArgs& a, cudaStream_t st, int ncomp) {
    const void* k = inv ? (const void*)xline8_kernel<true, C, PAIR> : (const void*)xline8_kernel<false, C, PAIR>;
    static bool attr[2] = {false, false};
    if (!attr[inv]) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XLine8<C>::smem);
      if (e != cudaSuccess) return e;
      attr[inv] = true;
    }
    if (a.ycount && (a.ycount % C || a.ybeg % C || a.ybeg < 0 || a.ybeg + a.ycount > N)) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SArgs*>(&a)};
    const int tiles = a.ycount ? a.ycount * ((N / 2) / C) + a.ycount / C : N * ((N / 2) / C) + N / C;
    // pairs: the two CTAs of a tile on adjacent block indices; single fields: components along y
    const dim3 grid = PAIR ? dim3(2 * tiles) : dim3(tiles, ncomp);
    return cudaLaunchKernel(k, grid, dim3(XLine8<C>::T), args, XLine8<C>::smem, st);
  }
  static cudaError_t xlaunch(bool inv, const SArgs& a, cudaStream_t st, int ncomp, bool pair) {
    if constexpr (N == 512) {
      if (pair) return a.narrow ? xlaunch_c<8, true>(inv, a, st, ncomp) : xlaunch_c<16, true>(inv, a, st, ncomp);
      return xlaunch_c<16, false>(inv, a, st, ncomp);
    }
    return cudaErrorInvalidValue;
  }


  static cudaError_t spass(int mode, int nc, int axis, const SArgs& a, cudaStream_t st) {
    if (nc < 1 || nc > 3) return cudaErrorInvalidValue;
    // plain passes: one component per CTA, components along gridDim.y
    if (mode == S_FWD && axis == AX_Y) return slaunch<S_FWD, 1, AX_Y>(a, st, nc);
    if (mode == S_INV && axis == AX_Y) return slaunch<S_INV, 1, AX_Y>(a, st, nc);
    if constexpr (N == 512) {
      // the vector x passes next to the register-fused k-space passes carry their representation
      if ((mode == S_FWD || mode == S_INV) && axis == AX_X && !a.generic && nc == 3)
        return xlaunch(mode == S_INV, a, st, nc, true);
      if ((mode == S_FWD || mode == S_INV) && axis == AX_X && !a.narrow && !a.generic)
        return xlaunch(mode == S_INV, a, st, nc, false);
    }
    if (mode == S_FWD && axis == AX_X)
      return a.narrow ? slaunch<S_FWD, 1, AX_X, 1>(a, st, nc) : slaunch<S_FWD, 1, AX_X>(a, st, nc);
    if (mode == S_INV && axis == AX_X)
      return a.narrow ? slaunch<S_INV, 1, AX_X, 1>(a, st, nc) : slaunch<S_INV, 1, AX_X>(a, st, nc);
    if constexpr (N == 512) {
      if (mode == S_DELTA && axis == AX_Y && !a.generic) return dlaunch(a, st);
    }
    if (mode == S_DELTA && axis == AX_Y) return slaunch<S_DELTA, 1, AX_Y>(a, st, 1);
    if (mode == S_ITER && axis == AX_Y && nc == 3) {
      if constexpr (N == 512) {
        if (!a.generic) return klaunch(a, st);
      }
      return slaunch<S_ITER, 3, AX_Y>(a, st, 1);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t build_tables(const float2* tw, float2* tabS, float2* tabZ, cudaStream_t st) {
    build_tables_kernel<N><<<4, 256, 0, st>>>(tw, tabS, tabZ);
    return cudaGetLastError();
  }

  static const MeshKernels* table() {
    static const MeshKernels t = {N, kZBlocks, kSBlocks, Plan<N>::kTab, Plan<N / 2>::kTab, N == 512 ? 1 : 0,
                                  &zpass, &spass, &build_tables};
    return &t;
  }
};

}  // namespace RG_KNS
}  // namespace rg
