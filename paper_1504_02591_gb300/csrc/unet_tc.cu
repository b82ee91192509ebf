// unet_tc.cu: periodic 3x3x3 convolution forward on the fifth-generation tensor cores (tcgen05).
//
// One CTA of 256 threads owns bx x by voxel tiles (runs of zlen voxels along z) and loops over its
// share of the grid's blocks (persistent grid).  Warps 0-2 are producers: for every chunk of input
// channel groups they stage the tiles' halo and the chunk's weight tiles in shared memory with
// 16-byte cp.async copies (two stages, so the next chunk loads while the tensor cores work on the
// current one).  One elected thread of warp 3 issues the chunk's MMAs, each reading its activation
// operand straight out of the halo through a shared-memory descriptor at the tap's offset, and
// commits them to the stage's mbarrier.  Accumulators live in tensor memory (one column block per
// tile, two buffers); after the last chunk of a block the four epilogue warps 4-7 read them back
// with tcgen05.ld (epilogue warp w owns TMEM lanes 32w..32w+31), add the bias, apply ReLU, round to
// bf16 and store channels-last (or, for the last layer, apply the 1x1 head and the residual and
// store float32).  Every wait on an mbarrier gives up after a bounded time, sets the
// caller's error flag, drains what is in flight and frees the tensor memory before returning.
#include "unet_tc.h"

#include <cstdint>

namespace rg {
namespace tc {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kThreads = 256;       // warps 0-2 producers, warp 3 MMA issue, warps 4-7 epilogue
constexpr int kProducers = 96;
constexpr int kStages = 2;
constexpr int kCtlBytes = 1536;     // mbarriers, TMEM slot, abort flag, offset tables, bias, head weights
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Bounded wait that also gives up as soon as another role of the CTA has given up.  Waiters off
// the critical path back off with nanosleep so they do not take issue slots from the MMA thread.
template <bool BACKOFF>
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
#pragma unroll 1
  for (int k = 0; k < 32; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
#pragma unroll 1
  for (long long it = 0; it < kWaitSpins; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kWaitNs) break;
    }
    if (BACKOFF) __nanosleep(128);
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

// Warp roles: warps 0-2 stage halos and weight tiles (two stages), warp 3 issues the MMAs (one
// thread), warps 4-7 run the epilogue (warp 4 + q reads TMEM lanes 32q..32q+31).  Two accumulator
// buffers in tensor memory let the epilogue of one block run under the MMAs of the next.
// Barriers: full[s] (producers -> MMA), empty[s] (MMA commit -> producers), accf[b] (MMA commit ->
// epilogue), acce[b] (epilogue -> MMA).
template <int ORIENT, int MODE, int NT>
__global__ void __launch_bounds__(kThreads, 1) tc_conv_kernel(const KArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned stage_bytes = a.halo_bytes + a.wts_bytes;
  unsigned char* ctl = sm + kStages * stage_bytes;
  const uint32_t ctl_a = smem_u32(ctl);
  const uint32_t bar_full = ctl_a, bar_empty = ctl_a + 16u, bar_accf = ctl_a + 32u, bar_acce = ctl_a + 48u;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 64);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 68);
  uint32_t* tapoff = reinterpret_cast<uint32_t*>(ctl + 128);   // per MMA: halo offset of its tap (16-B units)
  uint32_t* tileoff = reinterpret_cast<uint32_t*>(ctl + 256);  // per tile: halo offset of its run (16-B units)
  float* sbias = reinterpret_cast<float*>(ctl + 384);          // up to 128
  float* shead = reinterpret_cast<float*>(ctl + 896);          // up to 128
  const int HX = a.bx + 2, HY = a.by + 2;
  constexpr int ntiles = NT;   // = a.bx * a.by
  if (tid < a.nmma) {
    int dx, dy, dz;
    if (MODE == 0) {
      dx = tid / 9 - 1;
      dy = (tid / 3) % 3 - 1;
      dz = tid % 3 - 1;
    } else {
      const int dxy = tid >> 1;
      dx = dxy / 3 - 1;
      dy = dxy % 3 - 1;
      dz = (tid & 1) ? 1 : -1;
    }
    tapoff[tid] = (uint32_t)(((1 + dx) * HY + (1 + dy)) * a.hz + (1 + dz));
  }
  if (tid < ntiles) tileoff[tid] = (uint32_t)(((tid / a.by) * HY + tid % a.by) * a.hz);
  if (tid < 128) {
    sbias[tid] = tid < a.cout ? a.bias[tid] : 0.f;
    shead[tid] = (a.yout && tid < a.cout) ? __bfloat162float(a.head_w[tid]) : 0.f;
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full + 8u * s, kProducers);
      mbar_init(bar_empty + 8u * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_accf + 8u * b, 1);
      mbar_init(bar_acce + 8u * b, 128);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int n = a.n, m = n >> 1;
  const int G0 = a.c0 >> 3;
  const uint32_t plane = (uint32_t)(HX * HY * a.hz * 16);
  const int n_mine = (int)blockIdx.x < a.nblocks ? (a.nblocks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_items = n_mine * a.nchunk;
  const uint32_t acc_cols = (uint32_t)(ntiles * a.N);

  if (warp < kProducers / 32) {
    // ---- producers: halo rows (one warp per (group, hx, hy) row, lanes along z) and weight tiles
    for (int i = 0; i < n_items; ++i) {
      const int s = i % kStages, u = i / kStages;
      if (u >= 1 && !wait_bar<true>(bar_empty + 8u * s, (uint32_t)((u - 1) & 1), abort_flag, a.err)) break;
      const int blk = (int)blockIdx.x + (i / a.nchunk) * (int)gridDim.x;
      const int c = i % a.nchunk;
      int xb, yb, zb;
      block_origin(a, blk, xb, yb, zb);
      const uint32_t hdst = smem_u32(sm + (size_t)s * stage_bytes);
      const int nrows = a.gpc * HX * HY;
      for (int row = warp; row < nrows; row += kProducers / 32) {
        const int hyi = row % HY;
        const int t = row / HY;
        const int hxi = t % HX, gl = t / HX;
        const int g = c * a.gpc + gl;
        const int x = wrapc(xb - 1 + hxi, n), y = wrapc(yb - 1 + hyi, n);
        const bf16* base;
        int zstride, zshift;
        if (g < G0) {
          zstride = a.c0;
          if (a.up0) {
            base = a.src0 + ((long long)(x >> 1) * m + (y >> 1)) * m * a.c0 + g * 8;
            zshift = 1;
          } else {
            base = a.src0 + ((long long)x * n + y) * n * a.c0 + g * 8;
            zshift = 0;
          }
        } else {
          zstride = a.c1;
          zshift = 0;
          base = a.src1 + ((long long)x * n + y) * n * a.c1 + (g - G0) * 8;
        }
        const uint32_t drow = hdst + (uint32_t)(row * a.hz) * 16u;
        for (int hzi = lane; hzi < a.hz; hzi += 32) {
          const int z = wrapc(zb - 1 + hzi, n);
          cp_async16(drow + (uint32_t)hzi * 16u, base + (long long)(z >> zshift) * zstride);
        }
      }
      const uint32_t wdst = hdst + a.halo_bytes;
      const bf16* wsrc = a.wpack + (size_t)c * a.nmma * a.rows * 16;
      const int nw = a.nmma * a.rows * 2;
      for (int e = tid; e < nw; e += kProducers) cp_async16(wdst + (uint32_t)e * 16u, wsrc + (size_t)e * 8);
      cp_async_commit();
      cp_async_wait<0>();
      fence_proxy_async();      // make the copies visible to the tensor cores' (async-proxy) reads
      mbar_arrive(bar_full + 8u * s);
    }
    cp_async_wait<0>();
  } else if (warp == kProducers / 32) {
    // ---- one thread issues every MMA of the CTA
    if (lane == 0) {
      uint32_t toff[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) toff[j] = tileoff[j];
      int last = -1;
      for (int i = 0; i < n_items; ++i) {
        const int s = i % kStages, u = i / kStages;
        const int k = i / a.nchunk, c = i % a.nchunk, b = k & 1, ub = k >> 1;
        if (!wait_bar<false>(bar_full + 8u * s, (uint32_t)(u & 1), abort_flag, a.err)) break;
        if (c == 0 && ub >= 1 && !wait_bar<false>(bar_acce + 8u * b, (uint32_t)((ub - 1) & 1), abort_flag, a.err))
          break;
        tc_fence_after();
        const uint32_t hb = smem_u32(sm + (size_t)s * stage_bytes), wb = hb + a.halo_bytes;
        // the start-address field is the low 14 bits of the descriptor (address / 16, below 256 KB),
        // so operand offsets are added to a base descriptor directly
        const uint64_t a0 = smem_desc(hb, MODE == 0 ? plane : 16u, 128u);
        const uint64_t w0 = smem_desc(wb, 128u, 256u);
        const uint32_t wstep = (uint32_t)(a.rows * 32) >> 4;
        const uint32_t dbase = tmem + (uint32_t)b * acc_cols;
        for (int mm = 0; mm < a.nmma; ++mm) {
          const uint64_t wdesc = w0 + (uint64_t)(mm * wstep);
          const uint64_t at = a0 + tapoff[mm];
          const uint32_t accumulate = (c > 0 || mm > 0) ? 1u : 0u;
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            const uint64_t adesc = at + toff[j];
            if (ORIENT == 0)
              mma_bf16(dbase + (uint32_t)(j * a.N), adesc, wdesc, a.idesc, accumulate);
            else
              mma_bf16(dbase + (uint32_t)(j * a.N), wdesc, adesc, a.idesc, accumulate);
          }
        }
        mma_commit(bar_empty + 8u * s);
        if (c == a.nchunk - 1) mma_commit(bar_accf + 8u * b);
        last = i;
      }
      // every MMA issued must be complete before the tensor memory is released
      if (last >= 0)
        wait_bar<false>(bar_empty + 8u * (last % kStages), (uint32_t)((last / kStages) & 1), abort_flag, a.err);
    }
    __syncwarp();
  } else {
    // ---- epilogue: TMEM -> bias, ReLU, bf16 -> global (or the fused head)
    const int q = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    for (int k = 0; k < n_mine; ++k) {
      const int b = k & 1, ub = k >> 1;
      if (!wait_bar<true>(bar_accf + 8u * b, (uint32_t)(ub & 1), abort_flag, a.err)) break;
      tc_fence_after();
      const int blk = (int)blockIdx.x + k * (int)gridDim.x;
      int xb, yb, zb;
      block_origin(a, blk, xb, yb, zb);
      const uint32_t cbase = lane_base + (uint32_t)b * acc_cols;
      if (ORIENT == 0) {
        const int r = 32 * q + lane;   // voxel along the z run
#pragma unroll 1
        for (int j = 0; j < NT; ++j) {
          const int x = xb + j / a.by, y = yb + j % a.by, z = zb + r;
          const long long v = ((long long)x * n + y) * n + z;
          const float rv = a.yout ? a.res[v * a.res_stride] : 0.f;
          float hsum = 0.f;
          for (int cc = 0; cc < a.N; cc += 16) {
            float acc[16];
            tmem_ld16(cbase + (uint32_t)(j * a.N + cc), acc);
            __align__(16) bf16 o[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              o[e] = __float2bfloat16_rn(fmaxf(acc[e] + sbias[cc + e], 0.f));
              hsum = fmaf(__bfloat162float(o[e]), shead[cc + e], hsum);
            }
            if (!a.yout) {
#pragma unroll
              for (int h = 0; h < 2; ++h)
                if (cc + 8 * h < a.cout)
                  *reinterpret_cast<uint4*>(a.out + v * a.cout + cc + 8 * h) = *reinterpret_cast<const uint4*>(o + 8 * h);
            }
          }
          if (a.yout) a.yout[v] = a.head_b[0] + hsum + rv;
        }
      } else if (32 * q < a.cout) {
        const int co = 32 * q + lane;   // output channel = TMEM lane
        const bool valid = co < a.cout;
        const float bco = sbias[co < 128 ? co : 0];
        for (int j = 0; j < ntiles; ++j) {
          const int x = xb + j / a.by, y = yb + j % a.by;
          const long long v0 = ((long long)x * n + y) * n + zb;
          for (int cc = 0; cc < a.N; cc += 16) {
            float acc[16];
            tmem_ld16(cbase + (uint32_t)(j * a.N + cc), acc);
            if (valid) {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                a.out[(v0 + cc + e) * a.cout + co] = __float2bfloat16_rn(fmaxf(acc[e] + bco, 0.f));
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(bar_acce + 8u * b);
    }
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

template <int O, int M, int NT>
cudaError_t launch(const ConvPlan& p, const KArgs& a, cudaStream_t st) {
  const void* k = (const void*)tc_conv_kernel<O, M, NT>;
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
  tc_conv_kernel<O, M, NT><<<grid, kThreads, p.smem, st>>>(a);
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
    const int cols = 2 * bx * by * q.N;    // two accumulator buffers
    if (cols > 512) continue;
    const size_t halo = (size_t)q.gpc * (bx + 2) * (by + 2) * q.hz * 16;
    const size_t smem = kStages * (halo + q.wts_bytes) + kCtlBytes;
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
  const int nt = p.bx * p.by;
#define TC_NT(O_, M_)                                                  \
  switch (nt) {                                                       \
    case 16: return launch<O_, M_, 16>(p, a, st);                     \
    case 8: return launch<O_, M_, 8>(p, a, st);                       \
    case 4: return launch<O_, M_, 4>(p, a, st);                       \
    case 2: return launch<O_, M_, 2>(p, a, st);                       \
    case 1: return launch<O_, M_, 1>(p, a, st);                       \
    default: return cudaErrorInvalidValue;                            \
  }
  if (p.orient == 0) {
    if (p.mode == 0) TC_NT(0, 0) else TC_NT(0, 1)
  }
  if (p.mode == 0) TC_NT(1, 0) else TC_NT(1, 1)
#undef TC_NT
}

}  // namespace tc
}  // namespace rg
