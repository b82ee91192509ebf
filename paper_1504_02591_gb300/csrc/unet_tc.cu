// unet_tc.cu: periodic 3x3x3 convolution forward on the fifth-generation tensor cores (tcgen05).
//
// One CTA of 128 threads owns bx x by voxel tiles (runs of zlen voxels along z) and loops over its
// share of the grid's blocks (persistent grid).  For every chunk of input channel groups, all
// threads stage the tiles' halo and the chunk's weight tiles in shared memory with 16-byte cp.async
// copies (two stages, so the next chunk loads while the tensor cores work on the current one); one
// thread then issues the chunk's MMAs, each reading its activation operand straight out of the halo
// through a shared-memory descriptor at the tap's offset, and commits them to the stage's mbarrier.
// Accumulators live in tensor memory (one column block per tile); after the last chunk of a block
// the four warps read them back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), add the bias,
// apply ReLU, round to bf16 and store channels-last (or, for the last layer, apply the 1x1 head and
// the residual and store float32).  Every wait on an mbarrier gives up after a bounded time, sets the
// caller's error flag, drains what is in flight and frees the tensor memory before returning.
#include "unet_tc.h"

#include <cstdint>

namespace rg {
namespace tc {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kThreads = 128;
constexpr int kMaxSmem = 232448;                      // 227 KB per CTA
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait
constexpr long long kWaitSpins = 1ll << 26;

__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Waits for the completion of the mbarrier phase with the given parity; false after the time limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (long long it = 0; it < kWaitSpins; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// D (tmem) (+)= A (smem) x B (smem)^T, bf16 inputs, f32 accumulate; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on the mbarrier once every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane (the warp's 32-lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle (8-row x 16-byte core matrices): start address,
// leading byte offset (between the two core matrices along K), stride byte offset (between 8-row
// groups along M or N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major, M x N.
constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct KArgs {
  const bf16* src0;
  const bf16* src1;
  const bf16* wpack;
  const float* bias;
  bf16* out;
  const bf16* head_w;
  const float* head_b;
  const float* res;
  float* yout;
  int* err;
  int res_stride;
  int n, c0, up0, c1, cout;
  int gpc, nchunk, nmma, rows, N;
  int zlen, hz, bx, by;
  int tmem_cols;
  unsigned halo_bytes, wts_bytes;
  int nblocks, nbx, nby, nbz;
  uint32_t idesc;
};

__device__ __forceinline__ void block_origin(const KArgs& a, int blk, int& xb, int& yb, int& zb) {
  const int bz = blk % a.nbz;
  const int t = blk / a.nbz;
  const int by = t % a.nby, bx = t / a.nby;
  xb = bx * a.bx;
  yb = by * a.by;
  zb = bz * a.zlen;
}

template <int ORIENT, int MODE>
__global__ void __launch_bounds__(kThreads, 1) tc_conv_kernel(const KArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned stage_bytes = a.halo_bytes + a.wts_bytes;
  unsigned char* ctl = sm + 2 * stage_bytes;
  const uint32_t bar[2] = {smem_u32(ctl), smem_u32(ctl) + 8u};
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 16);
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar[0], 1);
    mbar_init(bar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int HX = a.bx + 2, HY = a.by + 2;
  const int ntiles = a.bx * a.by;
  const int n = a.n, m = n >> 1;
  const int G0 = a.c0 >> 3;
  const uint32_t plane = (uint32_t)(HX * HY * a.hz * 16);
  const int n_mine = (int)blockIdx.x < a.nblocks ? (a.nblocks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_items = n_mine * a.nchunk;

  // stage the halo of one (block, chunk) item and its weight tiles into stage s
  auto load = [&](int item, int s) {
    const int blk = (int)blockIdx.x + (item / a.nchunk) * (int)gridDim.x;
    const int c = item % a.nchunk;
    int xb, yb, zb;
    block_origin(a, blk, xb, yb, zb);
    const uint32_t hdst = smem_u32(sm + (size_t)s * stage_bytes);
    const int total = a.gpc * HX * HY * a.hz;
    for (int idx = tid; idx < total; idx += kThreads) {
      // layout [group][hx][hy][hz], 16 bytes (8 channels) per entry: the entry index is idx
      const int hzi = idx % a.hz;
      int t = idx / a.hz;
      const int hyi = t % HY;
      t /= HY;
      const int hxi = t % HX, gl = t / HX;
      const int g = c * a.gpc + gl;
      const int x = wrapc(xb - 1 + hxi, n), y = wrapc(yb - 1 + hyi, n), z = wrapc(zb - 1 + hzi, n);
      const bf16* src;
      if (g < G0) {
        if (a.up0)
          src = a.src0 + ((((long long)(x >> 1) * m + (y >> 1)) * m + (z >> 1)) * a.c0 + g * 8);
        else
          src = a.src0 + ((((long long)x * n + y) * n + z) * a.c0 + g * 8);
      } else {
        src = a.src1 + ((((long long)x * n + y) * n + z) * a.c1 + (g - G0) * 8);
      }
      cp_async16(hdst + (uint32_t)idx * 16u, src);
    }
    const uint32_t wdst = hdst + a.halo_bytes;
    const bf16* wsrc = a.wpack + (size_t)c * a.nmma * a.rows * 16;
    const int nw = a.nmma * a.rows * 2;
    for (int e = tid; e < nw; e += kThreads) cp_async16(wdst + (uint32_t)e * 16u, wsrc + (size_t)e * 8);
    cp_async_commit();
  };

  int ok = 1;
  int last_commit[2] = {-1, -1};
  if (n_items > 0) load(0, 0);
  for (int i = 0; i < n_items; ++i) {
    const int s = i & 1;
    if (i + 1 < n_items) {
      // stage s^1 was last read by the MMAs of item i-1
      int bad = 0;
      if (i >= 1) bad = !mbar_wait(bar[s ^ 1], (uint32_t)(((i - 1) >> 1) & 1));
      if (__syncthreads_or(bad)) {
        ok = 0;
        break;
      }
      load(i + 1, s ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    fence_proxy_async();
    __syncthreads();
    const int blk = (int)blockIdx.x + (i / a.nchunk) * (int)gridDim.x;
    const int c = i % a.nchunk;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t hb = smem_u32(sm + (size_t)s * stage_bytes), wb = hb + a.halo_bytes;
      const uint32_t lbo_act = MODE == 0 ? plane : 16u;
      for (int mm = 0; mm < a.nmma; ++mm) {
        int dx, dy, dz;
        if (MODE == 0) {
          dx = mm / 9 - 1;
          dy = (mm / 3) % 3 - 1;
          dz = mm % 3 - 1;
        } else {
          const int dxy = mm >> 1;
          dx = dxy / 3 - 1;
          dy = dxy % 3 - 1;
          dz = (mm & 1) ? 1 : -1;
        }
        const uint32_t tap = (uint32_t)((((1 + dx) * HY + (1 + dy)) * a.hz + (1 + dz)) * 16);
        const uint64_t wdesc = smem_desc(wb + (uint32_t)(mm * a.rows * 32), 128u, 256u);
        const uint32_t accumulate = (c > 0 || mm > 0) ? 1u : 0u;
        for (int j = 0; j < ntiles; ++j) {
          const int tx = j / a.by, ty = j % a.by;
          const uint32_t toff = (uint32_t)((tx * HY + ty) * a.hz * 16);
          const uint64_t adesc = smem_desc(hb + tap + toff, lbo_act, 128u);
          if (ORIENT == 0)
            mma_bf16(tmem + (uint32_t)(j * a.N), adesc, wdesc, a.idesc, accumulate);
          else
            mma_bf16(tmem + (uint32_t)(j * a.N), wdesc, adesc, a.idesc, accumulate);
        }
      }
      mma_commit(bar[s]);
    }
    last_commit[s] = i;
    if (c == a.nchunk - 1) {
      const int bad = !mbar_wait(bar[s], (uint32_t)((i >> 1) & 1));
      if (__syncthreads_or(bad)) {
        ok = 0;
        break;
      }
      tc_fence_after();
      int xb, yb, zb;
      block_origin(a, blk, xb, yb, zb);
      const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
      if (ORIENT == 0) {
        const int r = 32 * warp + lane;   // voxel along the z run
        for (int j = 0; j < ntiles; ++j) {
          const int x = xb + j / a.by, y = yb + j % a.by, z = zb + r;
          const long long v = ((long long)x * n + y) * n + z;
          float hsum = 0.f;
          for (int cc = 0; cc < a.N; cc += 16) {
            float acc[16];
            tmem_ld16(lane_base + (uint32_t)(j * a.N + cc), acc);
            __align__(16) bf16 o[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int co = cc + e;
              const float val = co < a.cout ? fmaxf(acc[e] + a.bias[co], 0.f) : 0.f;
              o[e] = __float2bfloat16_rn(val);
              if (a.yout && co < a.cout) hsum = fmaf(__bfloat162float(o[e]), __bfloat162float(a.head_w[co]), hsum);
            }
            if (!a.yout) {
#pragma unroll
              for (int h = 0; h < 2; ++h)
                if (cc + 8 * h < a.cout)
                  *reinterpret_cast<uint4*>(a.out + v * a.cout + cc + 8 * h) = *reinterpret_cast<const uint4*>(o + 8 * h);
            }
          }
          if (a.yout) a.yout[v] = a.head_b[0] + hsum + a.res[v * a.res_stride];
        }
      } else if (32 * warp < a.cout) {
        const int co = 32 * warp + lane;   // output channel = TMEM lane
        const bool valid = co < a.cout;
        const float b = valid ? a.bias[co] : 0.f;
        for (int j = 0; j < ntiles; ++j) {
          const int x = xb + j / a.by, y = yb + j % a.by;
          const long long v0 = ((long long)x * n + y) * n + zb;
          for (int cc = 0; cc < a.N; cc += 16) {
            float acc[16];
            tmem_ld16(lane_base + (uint32_t)(j * a.N + cc), acc);
            if (valid) {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                a.out[(v0 + cc + e) * a.cout + co] = __float2bfloat16_rn(fmaxf(acc[e] + b, 0.f));
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  cp_async_wait<0>();
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // let every MMA already issued finish (bounded) before the tensor memory is released
    for (int s = 0; s < 2; ++s)
      if (last_commit[s] >= 0) mbar_wait(bar[s], (uint32_t)((last_commit[s] >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
  }
}

// out[c][m][row][kg][e] (the shared-memory image: core matrix (row/8, kg) at row/8*256 + kg*128 bytes)
__global__ void pack_kernel(const bf16* __restrict__ w, int cin, int cout, int mode, int nchunk, int nmma, int rows,
                            bf16* __restrict__ out) {
  const long long total = (long long)nchunk * nmma * rows * 16;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i & 7), kg = (int)((i >> 3) & 1);
    const long long q = i >> 4;
    const int r = (int)(q % rows);
    const int mm = (int)((q / rows) % nmma);
    const int c = (int)(q / rows / nmma);
    int tap, ci;
    bool valid = true;
    if (mode == 0) {
      tap = mm;
      ci = (2 * c + kg) * 8 + e;
    } else {
      const int dxy = mm >> 1;
      const int dzi = (mm & 1) ? 2 + kg : kg;   // dz + 1 of this K half; 3 is the zero tap dz = +2
      valid = dzi < 3;
      tap = dxy * 3 + dzi;
      ci = c * 8 + e;
    }
    bf16 val = __float2bfloat16_rn(0.f);
    if (valid && ci < cin && r < cout) val = w[((size_t)tap * cin + ci) * cout + r];
    const size_t o = ((size_t)c * nmma + mm) * rows * 16 + (size_t)(r >> 3) * 128 + kg * 64 + (r & 7) * 8 + e;
    out[o] = val;
  }
}

template <int O, int M>
cudaError_t launch(const ConvPlan& p, const KArgs& a, cudaStream_t st) {
  const void* k = (const void*)tc_conv_kernel<O, M>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  if (e != cudaSuccess) return e;
  int occ = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, p.smem);
  if (e != cudaSuccess) return e;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tm = 512 / p.tmem_cols;      // CTAs whose tensor memory fits on one SM together
  if (occ > tm) occ = tm;
  if (occ < 1) occ = 1;
  const int grid = p.nblocks < sms * occ ? p.nblocks : sms * occ;
  tc_conv_kernel<O, M><<<grid, kThreads, p.smem, st>>>(a);
  return cudaGetLastError();
}

size_t round_up(size_t v, size_t q) { return (v + q - 1) / q * q; }

}  // namespace

bool plan_conv(int n, int c0, int up0, int c1, int cin, int cout, ConvPlan* out) {
  ConvPlan q;
  if (c0 <= 0 || c0 % 8 || c1 < 0 || c1 % 8 || cout < 8 || cout % 8 || cout > 128 || cin > c0 + c1) return false;
  if (n % 128 == 0) {
    q.orient = 0;
    q.zlen = 128;
  } else if (n == 64) {
    q.orient = 1;
    q.zlen = 64;
  } else {
    return false;
  }
  q.n = n;
  q.c0 = c0;
  q.up0 = up0 ? 1 : 0;
  q.c1 = c1;
  q.cin = cin;
  q.cout = cout;
  const int G = (c0 + c1) / 8;
  q.mode = (G % 2 == 0) ? 0 : 1;
  q.gpc = q.mode == 0 ? 2 : 1;
  q.nchunk = G / q.gpc;
  q.nmma = q.mode == 0 ? 27 : 18;
  if (q.orient == 0) {
    q.N = (cout + 15) / 16 * 16;
    q.rows = q.N;
  } else {
    q.N = q.zlen;
    q.rows = cout;
  }
  q.hz = q.zlen + 4;
  // orient 1 reads 128 weight rows per MMA: the rows past cout run into the next tiles (their
  // products land in TMEM lanes that are never read), and past the last tile into this padding
  q.wts_bytes = round_up((size_t)q.nmma * q.rows * 32 + (q.orient == 1 ? (size_t)(128 - cout) * 32 : 0), 128);
  static const int cand[][2] = {{4, 4}, {2, 4}, {4, 2}, {2, 2}, {1, 2}, {2, 1}, {1, 1}};
  bool found = false;
  for (const auto& c : cand) {
    const int bx = c[0], by = c[1];
    if (n % bx || n % by) continue;
    const int cols = bx * by * q.N;
    if (cols > 512) continue;
    const size_t halo = (size_t)q.gpc * (bx + 2) * (by + 2) * q.hz * 16;
    const size_t smem = 2 * (halo + q.wts_bytes) + 64;
    if (smem > (size_t)kMaxSmem) continue;
    q.bx = bx;
    q.by = by;
    q.halo_bytes = halo;
    q.smem = smem;
    int tc = 32;
    while (tc < cols) tc *= 2;
    q.tmem_cols = tc;
    found = true;
    break;
  }
  if (!found) return false;
  q.nblocks = (n / q.bx) * (n / q.by) * (n / q.zlen);
  q.packed_elems = (size_t)q.nchunk * q.nmma * q.rows * 16;
  *out = q;
  return true;
}

cudaError_t pack_weights(const ConvPlan& p, const bf16* w, bf16* out, cudaStream_t st) {
  const long long total = (long long)p.packed_elems;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  pack_kernel<<<blocks, 256, 0, st>>>(w, p.cin, p.cout, p.mode, p.nchunk, p.nmma, p.rows, out);
  return cudaGetLastError();
}

cudaError_t conv_forward(const ConvPlan& p, const ConvIO& io, cudaStream_t st) {
  KArgs a;
  a.src0 = io.src0;
  a.src1 = io.src1;
  a.wpack = io.wpack;
  a.bias = io.bias;
  a.out = io.out;
  a.head_w = io.head_w;
  a.head_b = io.head_b;
  a.res = io.res;
  a.yout = io.yout;
  a.err = io.err;
  a.res_stride = io.res_stride;
  a.n = p.n;
  a.c0 = p.c0;
  a.up0 = p.up0;
  a.c1 = p.c1;
  a.cout = p.cout;
  a.gpc = p.gpc;
  a.nchunk = p.nchunk;
  a.nmma = p.nmma;
  a.rows = p.rows;
  a.N = p.N;
  a.zlen = p.zlen;
  a.hz = p.hz;
  a.bx = p.bx;
  a.by = p.by;
  a.tmem_cols = p.tmem_cols;
  a.halo_bytes = (unsigned)p.halo_bytes;
  a.wts_bytes = (unsigned)p.wts_bytes;
  a.nblocks = p.nblocks;
  a.nbx = p.n / p.bx;
  a.nby = p.n / p.by;
  a.nbz = p.n / p.zlen;
  a.idesc = instr_desc(128, p.N);
  if (!a.err || !a.wpack || !a.bias || !a.src0 || (p.c1 && !a.src1)) return cudaErrorInvalidValue;
  if (io.yout && (p.orient != 0 || !io.head_w || !io.head_b || !io.res)) return cudaErrorInvalidValue;
  if (!io.yout && !io.out) return cudaErrorInvalidValue;
  if (p.orient == 0) return p.mode == 0 ? launch<0, 0>(p, a, st) : launch<0, 1>(p, a, st);
  return p.mode == 0 ? launch<1, 0>(p, a, st) : launch<1, 1>(p, a, st);
}

}  // namespace tc
}  // namespace rg
