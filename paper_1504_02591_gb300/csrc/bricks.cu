// bricks.cu: brick-sorted particle pipeline for the CIC deposit and the reconstruction shift.
//
// Particles are packed into 16-byte records (per axis: node index << 21 | 21-bit fraction of a cell,
// rounded down; then the weight) and counting-sorted by their 8^3-cell brick.  The deposit
// then gives each brick to one warp, which accumulates the CIC weights (Sec. 3 mass assignment,
// here cloud-in-cell) of its particles into a 9^3 node tile in shared memory and flushes the tile
// with one global atomic per non-zero node.  The shift (Sec. 1, reversing Eq. Lagrange) stages the
// brick's 9^3 nodes of the three Psi components in shared memory and interpolates every particle of
// the brick from there; results go back to the catalogue's own order through the sort permutation.
#include "bricks.h"

namespace rg {

namespace {

constexpr int kWarps = 8;                 // warps per CTA in the brick kernels
constexpr uint32_t kFracOne = 1u << kFracBits;
constexpr uint32_t kFracMask = kFracOne - 1;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Node index and 21-bit fraction of a grid coordinate u, from t = u 2^21 (computed as x times
// scale 2^21: the same rounding as u itself).  T = floor(t); node = T >> 21 = floor(u)
// (arithmetic shift, also for negative u), fraction = T mod 2^21.  Rounding down keeps a point just
// below the periodic boundary on its own side (its image stays below L, where its line of sight
// points).  Two float64 operations per axis: float64 runs at a small fraction of the float32 rate
// on this GPU.
__device__ __forceinline__ uint32_t pack_axis(double t, int n) {
  const long long T = __double2ll_rd(t);
  int c = (int)(T >> kFracBits);
  if (c < 0 || c >= n) c = ((c % n) + n) % n;   // outside [0, L): periodic image
  return ((uint32_t)c << kFracBits) | (uint32_t)(T & (long long)kFracMask);
}

template <typename PT>
__device__ __forceinline__ void pack(const PT* __restrict__ pos, long long p, double scale21, int n,
                                     uint32_t (&q)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a] = pack_axis((double)pos[3 * p + a] * scale21, n);
}

__device__ __forceinline__ uint32_t brick_key(const uint32_t (&q)[3], int nb) {
  const uint32_t bx = (q[0] >> kFracBits) / kBrick, by = (q[1] >> kFracBits) / kBrick,
                 bz = (q[2] >> kFracBits) / kBrick;
  return (bx * (uint32_t)nb + by) * (uint32_t)nb + bz;
}

// Count particles per brick; each particle keeps its brick and its arrival rank in the brick.  The
// positions (and weights) are read here only, once: each particle's packed record is kept in input
// order for the scatter.
template <typename PT>
__global__ void __launch_bounds__(256) count_kernel(const PT* __restrict__ pos, const float* __restrict__ w,
                                                    long long np, double scale, int n, int nb,
                                                    uint32_t* __restrict__ hist, uint32_t* __restrict__ key,
                                                    uint32_t* __restrict__ rank, uint4* __restrict__ pre) {
  const double scale21 = scale * (double)kFracOne;   // exact: a power of two
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    uint32_t q[3];
    pack(pos, p, scale21, n, q);
    const uint32_t k = brick_key(q, nb);
    key[p] = k;
    rank[p] = atomicAdd(hist + k, 1u);
    pre[p] = make_uint4(q[0], q[1], q[2], __float_as_uint(w ? w[p] : 1.f));
  }
}

// Place every particle's record at offs[brick] + rank.
__global__ void __launch_bounds__(256) scatter_kernel(const uint4* __restrict__ pre, long long np,
                                                      const uint32_t* __restrict__ offs, const uint32_t* __restrict__ key,
                                                      const uint32_t* __restrict__ rank, uint4* __restrict__ rec,
                                                      uint32_t* __restrict__ perm) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const uint32_t slot = offs[key[p]] + rank[p];
    rec[slot] = pre[p];
    perm[slot] = (uint32_t)p;
  }
}

// Exclusive scan of m counts: blocks of 1024 (256 threads x 4), then the block sums, then the add.
__global__ void __launch_bounds__(256) scan_blocks_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                          uint32_t* __restrict__ bsum, int m) {
  __shared__ uint32_t wsum[8];
  const int base = blockIdx.x * 1024 + threadIdx.x * 4;
  uint32_t v[4], s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = (base + j < m) ? in[base + j] : 0u;
    s += v[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t woff = 0, tot = 0;
  for (int i = 0; i < 8; ++i) {
    if (i < warp) woff += wsum[i];
    tot += wsum[i];
  }
  uint32_t run = woff + x - s;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < m) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t* __restrict__ bsum, int nblk, uint32_t* __restrict__ total) {
  __shared__ uint32_t wsum[32];
  const int base = threadIdx.x * 4;
  uint32_t v[4], s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = (base + j < nblk) ? bsum[base + j] : 0u;
    s += v[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t woff = 0, tot = 0;
  for (int i = 0; i < 32; ++i) {
    if (i < warp) woff += wsum[i];
    tot += wsum[i];
  }
  uint32_t run = woff + x - s;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < nblk) bsum[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(256) scan_add_kernel(uint32_t* __restrict__ out, const uint32_t* __restrict__ bsum,
                                                       int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] += bsum[i / 1024];
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kWarps * 32) deposit_kernel(const uint32_t* __restrict__ offs,
                                                              const uint4* __restrict__ rec, int n, int nb,
                                                              float* __restrict__ rho, double* __restrict__ partials) {
  __shared__ float tiles[kWarps][kBrickNodes];
  __shared__ double wsh[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* tile = tiles[warp];
  const int nb3 = nb * nb * nb;
  const float inv = 1.f / (float)kFracOne;
  double wsum = 0.0;
  for (int b = blockIdx.x * kWarps + warp; b < nb3; b += gridDim.x * kWarps) {
    const uint32_t s0 = offs[b], s1 = offs[b + 1];
    if (s0 == s1) continue;
    for (int j = lane; j < kBrickNodes; j += 32) tile[j] = 0.f;
    __syncwarp();
    const int ox = (b / (nb * nb)) * kBrick, oy = ((b / nb) % nb) * kBrick, oz = (b % nb) * kBrick;
    float bw = 0.f;   // this lane's weight in the brick (float64 once per brick, not per particle)
    for (uint32_t i = s0 + lane; i < s1; i += 32) {
      const uint4 r = rec[i];
      const float wv = __uint_as_float(r.w);
      bw += wv;
      const int lx = (int)(r.x >> kFracBits) - ox, ly = (int)(r.y >> kFracBits) - oy, lz = (int)(r.z >> kFracBits) - oz;
      const float tx = (float)(r.x & kFracMask) * inv, ty = (float)(r.y & kFracMask) * inv,
                  tz = (float)(r.z & kFracMask) * inv;
      const float wx0 = wv * (1.f - tx), wx1 = wv * tx, wy0 = 1.f - ty, wy1 = ty, wz0 = 1.f - tz, wz1 = tz;
      const int c = (lx * kBrickHalo + ly) * kBrickHalo + lz;
      constexpr int DY = kBrickHalo, DX = kBrickHalo * kBrickHalo;
      atomicAdd(tile + c, wx0 * wy0 * wz0);
      atomicAdd(tile + c + 1, wx0 * wy0 * wz1);
      atomicAdd(tile + c + DY, wx0 * wy1 * wz0);
      atomicAdd(tile + c + DY + 1, wx0 * wy1 * wz1);
      atomicAdd(tile + c + DX, wx1 * wy0 * wz0);
      atomicAdd(tile + c + DX + 1, wx1 * wy0 * wz1);
      atomicAdd(tile + c + DX + DY, wx1 * wy1 * wz0);
      atomicAdd(tile + c + DX + DY + 1, wx1 * wy1 * wz1);
    }
    wsum += bw;
    __syncwarp();
    for (int j = lane; j < kBrickNodes; j += 32) {
      const float v = tile[j];
      if (v != 0.f) {
        int gx = ox + j / (kBrickHalo * kBrickHalo), gy = oy + (j / kBrickHalo) % kBrickHalo, gz = oz + j % kBrickHalo;
        if (gx >= n) gx -= n;
        if (gy >= n) gy -= n;
        if (gz >= n) gz -= n;
        atomicAdd(rho + ((size_t)gx * n + gy) * n + gz, v);
      }
    }
    __syncwarp();
  }
  wsum = warp_sum_d(wsum);
  if (lane == 0) wsh[warp] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += wsh[i];
    partials[blockIdx.x] = s;
  }
}

template <typename PT>
__device__ __forceinline__ void write_pos(const BrickShiftArgs& a, uint32_t p, const float (&d)[3]) {
  const PT* pos = static_cast<const PT*>(a.pos);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double y = (double)pos[3 * (size_t)p + c] + d[c];
    if (a.periodic) {
      y -= floor(y / a.L) * a.L;
      if (y >= a.L) y -= a.L;
    }
    a.pos_out[3 * (size_t)p + c] = y;
  }
}

__global__ void __launch_bounds__(kWarps * 32) shift_kernel(const uint32_t* __restrict__ offs,
                                                            const uint4* __restrict__ rec,
                                                            const uint32_t* __restrict__ perm, int n, int nb,
                                                            const BrickShiftArgs a) {
  extern __shared__ float ssm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* tile = ssm + warp * 3 * kBrickNodes;
  const int nb3 = nb * nb * nb;
  const float inv = 1.f / (float)kFracOne;
  const float Hf = (float)a.H;
  for (int b = blockIdx.x * kWarps + warp; b < nb3; b += gridDim.x * kWarps) {
    const uint32_t s0 = offs[b], s1 = offs[b + 1];
    if (s0 == s1) continue;
    const int ox = (b / (nb * nb)) * kBrick, oy = ((b / nb) % nb) * kBrick, oz = (b % nb) * kBrick;
    for (int j = lane; j < kBrickNodes; j += 32) {
      int gx = ox + j / (kBrickHalo * kBrickHalo), gy = oy + (j / kBrickHalo) % kBrickHalo, gz = oz + j % kBrickHalo;
      if (gx >= n) gx -= n;
      if (gy >= n) gy -= n;
      if (gz >= n) gz -= n;
      const size_t g = ((size_t)gx * n + gy) * n + gz;
      tile[j] = __ldg(a.psi[0] + g);
      tile[kBrickNodes + j] = __ldg(a.psi[1] + g);
      tile[2 * kBrickNodes + j] = __ldg(a.psi[2] + g);
    }
    __syncwarp();
    for (uint32_t i = s0 + lane; i < s1; i += 32) {
      const uint4 r = rec[i];
      const int cx = (int)(r.x >> kFracBits), cy = (int)(r.y >> kFracBits), cz = (int)(r.z >> kFracBits);
      const float tx = (float)(r.x & kFracMask) * inv, ty = (float)(r.y & kFracMask) * inv,
                  tz = (float)(r.z & kFracMask) * inv;
      const int c = ((cx - ox) * kBrickHalo + (cy - oy)) * kBrickHalo + (cz - oz);
      constexpr int DY = kBrickHalo, DX = kBrickHalo * kBrickHalo;
      const float cw[8] = {(1.f - tx) * (1.f - ty) * (1.f - tz), (1.f - tx) * (1.f - ty) * tz,
                           (1.f - tx) * ty * (1.f - tz),         (1.f - tx) * ty * tz,
                           tx * (1.f - ty) * (1.f - tz),         tx * (1.f - ty) * tz,
                           tx * ty * (1.f - tz),                 tx * ty * tz};
      const int co[8] = {0, 1, DY, DY + 1, DX, DX + 1, DX + DY, DX + DY + 1};
      float ps[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = fmaf(cw[k], tile[q * kBrickNodes + c + co[k]], acc);
        ps[q] = acc;
      }
      float d[3];
      if (a.is_galaxy) {
        float rx, ry, rz;
        if (a.los_mode == 1) {
          rx = a.los.x; ry = a.los.y; rz = a.los.z;
        } else {
          const float dx = fmaf(tx, Hf, a.off[cx]), dy = fmaf(ty, Hf, a.off[n + cy]), dz = fmaf(tz, Hf, a.off[2 * n + cz]);
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
      const uint32_t p = perm[i];
      a.shift[3 * (size_t)p + 0] = d[0];
      a.shift[3 * (size_t)p + 1] = d[1];
      a.shift[3 * (size_t)p + 2] = d[2];
      if (a.pos_out) {
        if (a.dtype == 0) write_pos<double>(a, p, d);
        else write_pos<float>(a, p, d);
      }
    }
    __syncwarp();
  }
}

constexpr int kGrid = 152 * 8;

}  // namespace

size_t brick_scratch_bytes(int n) {
  const size_t nb3 = (size_t)(n / kBrick) * (n / kBrick) * (n / kBrick);
  const size_t ch = (size_t)sort_chunk(n);
  return a256(nb3 * 4) + a256((nb3 + 1) * 4) + a256(4096 * 4) + 2 * a256(ch * 16) + 3 * a256(ch * 4);
}

BrickBuffers brick_buffers(char* base, int n, double L) {
  BrickBuffers b{};
  b.n = n;
  b.nb = n / kBrick;
  b.scale = (double)n / L;
  b.chunk = sort_chunk(n);
  const size_t nb3 = (size_t)b.nb * b.nb * b.nb;
  const size_t ch = (size_t)b.chunk;
  b.hist = reinterpret_cast<uint32_t*>(base);
  base += a256(nb3 * 4);
  b.offs = reinterpret_cast<uint32_t*>(base);
  base += a256((nb3 + 1) * 4);
  b.bsum = reinterpret_cast<uint32_t*>(base);
  base += a256(4096 * 4);
  b.rec = reinterpret_cast<uint4*>(base);
  base += a256(ch * 16);
  b.perm = reinterpret_cast<uint32_t*>(base);
  base += a256(ch * 4);
  b.key = reinterpret_cast<uint32_t*>(base);
  base += a256(ch * 4);
  b.rank = reinterpret_cast<uint32_t*>(base);
  base += a256(ch * 4);
  b.pre = reinterpret_cast<uint4*>(base);
  return b;
}

int brick_grid() { return kGrid; }

cudaError_t brick_sort(const BrickBuffers& b, const void* pos, int dtype, const float* w, long long np, cudaStream_t st) {
  if (np <= 0 || np > b.chunk) return np == 0 ? cudaSuccess : cudaErrorInvalidValue;
  const int m = b.nb * b.nb * b.nb;
  const int nblk = (m + 1023) / 1024;
  if (nblk > 4096) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(b.hist, 0, (size_t)m * 4, st);
  if (e != cudaSuccess) return e;
  long long want = (np + 255) / 256;
  const int blocks = (int)(want < kGrid * 2 ? want : kGrid * 2);
  if (dtype == 0)
    count_kernel<double><<<blocks, 256, 0, st>>>((const double*)pos, w, np, b.scale, b.n, b.nb, b.hist, b.key, b.rank,
                                                  b.pre);
  else
    count_kernel<float><<<blocks, 256, 0, st>>>((const float*)pos, w, np, b.scale, b.n, b.nb, b.hist, b.key, b.rank,
                                                 b.pre);
  scan_blocks_kernel<<<nblk, 256, 0, st>>>(b.hist, b.offs, b.bsum, m);
  scan_sums_kernel<<<1, 1024, 0, st>>>(b.bsum, nblk, b.offs + m);
  scan_add_kernel<<<(m + 255) / 256 < kGrid ? (m + 255) / 256 : kGrid, 256, 0, st>>>(b.offs, b.bsum, m);
  scatter_kernel<<<blocks, 256, 0, st>>>(b.pre, np, b.offs, b.key, b.rank, b.rec, b.perm);
  return cudaGetLastError();
}

cudaError_t brick_deposit(const BrickBuffers& b, float* rho, double* partials, cudaStream_t st) {
  deposit_kernel<<<kGrid, kWarps * 32, 0, st>>>(b.offs, b.rec, b.n, b.nb, rho, partials);
  return cudaGetLastError();
}

cudaError_t brick_shift(const BrickBuffers& b, const BrickShiftArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(float) * kWarps * 3 * kBrickNodes;
  cudaError_t e = cudaFuncSetAttribute((const void*)shift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  shift_kernel<<<kGrid, kWarps * 32, smem, st>>>(b.offs, b.rec, b.perm, b.n, b.nb, a);
  return cudaGetLastError();
}

}  // namespace rg
