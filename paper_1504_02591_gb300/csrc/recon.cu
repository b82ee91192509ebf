// recon.cu: the C ABI (include/recon.h) and the host-side orchestration of the passes.
//
// Pipeline per reconstruction (Burden, Percival & Howlett 2015):
//   deposit  CIC of galaxies and randoms -> rho_g, rho_r; sums of weights (float64)
//   smooth   Gaussian exp(-k^2 R^2/2) as three periodic 1-D convolutions (x, y passes, then z
//            inside the next pass); Z: delta = rho_g,s/(alpha rho_r,s) - 1 in the mask (+ lognormal)
//            and its r2c | X                                                        (Sec. 3.1, 3.2)
//   iterate  Y: delta(k), S_-1 = delta/b, Psi_s = Z[delta/b] | X | Z: P_0 = (1-c)(Psi_s.r)r | X
//            repeat: Y: S_n = delta/b + beta i k.P_n, norms, Psi = i k S/k^2 | X |
//                    Z: P = (Psi.r)r (or the final real Psi) | X                  (Sec. 5.1)
//   shift    CIC interpolation of Psi to the particles, d = -(Psi + f (Psi.r) r) or -Psi (Sec. 1)
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/recon.h"
#include "batch_graph.h"
#include "bricks.h"
#include "cic.h"
#include "conv.h"
#include "diag.h"
#include "fd.h"
#include "loop.h"
#include "warm.h"
#include "types.h"

namespace rg {
const MeshKernels* mesh_kernels_32();
const MeshKernels* mesh_kernels_48();
const MeshKernels* mesh_kernels_64();
const MeshKernels* mesh_kernels_96();
const MeshKernels* mesh_kernels_128();
const MeshKernels* mesh_kernels_256();
const MeshKernels* mesh_kernels_384();
const MeshKernels* mesh_kernels_512();
const MeshKernels* mesh_kernels_1024();
const MeshKernels* mesh_kernels_256_order1();
const MeshKernels* mesh_kernels_384_order1();

// The kernels of mesh side n in radix order `order` (1: the alternative order, where one is built).
const MeshKernels* mesh_kernels_order(int n, int order) {
  if (order == 0) return mesh_kernels(n);
  if (order != 1) return nullptr;
  if (n == 256) return mesh_kernels_256_order1();
  if (n == 384) return mesh_kernels_384_order1();
  return nullptr;
}

const MeshKernels* mesh_kernels(int n) {
  switch (n) {
    case 32: return mesh_kernels_32();
    case 48: return mesh_kernels_48();
    case 64: return mesh_kernels_64();
    case 96: return mesh_kernels_96();
    case 128: return mesh_kernels_128();
    case 256: return mesh_kernels_256();
    case 384: return mesh_kernels_384();
    case 512: return mesh_kernels_512();
    case 1024: return mesh_kernels_1024();
    default: return nullptr;
  }
}
}  // namespace rg

using namespace rg;

namespace {

constexpr long long kStageParticles = 1LL << 21;   // particles per host<->device chunk
constexpr size_t kStageBytesPer = 64;              // 24 pos + 4 w + 12 shift + 24 pos_out

enum State { ST_CREATED = 0, ST_DEPOSITED = 1, ST_SMOOTHED = 2, ST_ITERATED = 3 };

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t field_M, field_Q, field, wfield, tw, tabs, tabz, off, taps, red, partials, stage, bricks, coarse, total;
};

Layout layout_for(int n) {
  const MeshKernels* mk = mesh_kernels(n);
  Layout l{};
  l.field_M = align256((size_t)n * n * n * sizeof(float));
  l.field_Q = align256((size_t)n * n * sizeof(float2));
  l.field = l.field_M + l.field_Q;
  l.wfield = mk->kspace_fused ? l.field : 0;   // register-fused path: Psi_z in C form (fourth vector field)
  l.tw = align256((size_t)n * sizeof(float2));
  // stage tables: room for either radix order (recon_set_option can switch)
  const MeshKernels* alt = mesh_kernels_order(n, 1);
  const int tab_s = alt && alt->tab_s > mk->tab_s ? alt->tab_s : mk->tab_s;
  const int tab_z = alt && alt->tab_z > mk->tab_z ? alt->tab_z : mk->tab_z;
  l.tabs = align256((size_t)tab_s * sizeof(float2) + 16);
  l.tabz = align256((size_t)tab_z * sizeof(float2) + 16);
  l.off = align256((size_t)3 * n * sizeof(float));
  l.taps = align256((size_t)n * sizeof(float));
  // reduction slots, the loop state, the finalize block sums and counter
  l.red = align256(64 * sizeof(double) + sizeof(LoopState) + kFinalizeBlocks * 4 * sizeof(double) + 64);
  size_t nb = (size_t)mk->z_blocks;
  if ((size_t)mk->s_blocks > nb) nb = mk->s_blocks;
  if ((size_t)kDepositBlocks > nb) nb = kDepositBlocks;
  if ((size_t)conv_blocks(n) > nb) nb = conv_blocks(n);
  if ((size_t)brick_grid() > nb) nb = brick_grid();
  l.partials = align256(nb * 4 * sizeof(double));
  l.stage = align256(2 * (size_t)kStageParticles * kStageBytesPer);   // two buffers (copy/compute overlap)
  l.bricks = align256(brick_scratch_bytes(n));
  l.coarse = align256((size_t)(n / 2) * (n / 2) * (n / 2) * sizeof(float));   // warm start, level >= 1
  l.total = 5 * l.field + l.wfield + l.tw + l.tabs + l.tabz + l.off + l.taps + l.red + l.partials + l.stage + l.bricks +
            l.coarse;
  return l;
}

bool valid_params(const recon_params* p) {
  if (!p) return false;
  const int n = p->nmesh[0];
  if (p->nmesh[1] != n || p->nmesh[2] != n) return false;
  if (!mesh_kernels(n)) return false;
  if (!(p->box[0] > 0) || p->box[1] != p->box[0] || p->box[2] != p->box[0]) return false;
  if (!(p->b > 0) || !std::isfinite(p->f) || p->f < 0) return false;
  if (!(p->smooth_R >= 0)) return false;
  if (p->los_mode != RECON_LOS_RADIAL && p->los_mode != RECON_LOS_FIXED) return false;
  if (p->los_mode == RECON_LOS_FIXED) {
    const double q = p->observer[0] * p->observer[0] + p->observer[1] * p->observer[1] +
                     p->observer[2] * p->observer[2];
    if (!(q > 0)) return false;
  }
  if (p->mean_density_mode != RECON_MEAN_RANDOMS && p->mean_density_mode != RECON_MEAN_UNIFORM) return false;
  if (!(p->mask_frac >= 0)) return false;
  return true;
}

}  // namespace

struct recon_handle {
  recon_params p{};
  int n = 0;
  double L = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  Layout lay{};
  Field V[3]{}, D{}, S{};
  Field W{};             // N = 512: Psi_z between the inverse x pass and the projection (C form)
  float2* tw = nullptr;
  float2* tabs = nullptr;   // stage twiddles, N-point plan
  float2* tabz = nullptr;   // stage twiddles, N/2-point plan
  float* off = nullptr;
  float* taps = nullptr;   // smoothing kernel g[t0 .. t0 + ntap - 1]
  int ntap = 1, t0 = 0;
  // the tables the passes read: the handle's own (taps, off) or a batch's per-mock copies
  const float* cur_taps = nullptr;
  const float* cur_off = nullptr;
  double* red = nullptr;
  LoopState* loop = nullptr;   // device-driven iteration state (inside the red region)
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  cudaStream_t copy_st = nullptr;      // host<->device copies of the staged shift (overlap the kernels)
  cudaEvent_t ev_in[2] = {}, ev_out[2] = {}, ev_free[2] = {};
  int use_graph = 1;
  double* partials = nullptr;
  double* fin_bsum = nullptr;          // finalize: per-block sums (inside the red region)
  unsigned int* fin_counter = nullptr; // finalize: blocks done (zero between launches)
  char* stage = nullptr;
  BrickBuffers bb{};       // brick sort of one particle chunk
  const MeshKernels* mk = nullptr;
  int state = ST_CREATED;
  int deposit_path = RECON_PATH_DIRECT;
  int shift_path = RECON_PATH_SORTED;
  int narrow_lines = 0;
  int kspace_generic = 0;
  int plane_batch = 0;   // register-fused path: y-planes per batch of the x -> z -> x passes (0: off)
  int assign = 0;        // mass assignment of the deposit: 0 CIC, 1 NGP (the paper's binning)
  int kiter_tma = 0;     // N = 512 fused path: 1 streams the source update's inputs by TMA
  int radix_order = 0;   // FFT plans: 0 default, 1 the alternative order (mk is that order's table)
  bool tmaps_ok = false; // its tensor maps were built
  KIterMaps tmaps{};
  int reuse_sort = 0;
  // the catalogue whose brick order the sort buffers hold (sorted deposit, one chunk)
  struct SortMemo {
    int valid;
    const void* pos;
    int64_t n;
    int dtype, on_device;
  } memo{};
  int d_is_k = 0;
  int delta_real_valid = 0;
  float* ucoarse = nullptr;   // block means of the start's radial displacement (warm start, level >= 1)
  int warm_level = -1;        // level of the pending warm start prepared by recon_start_features
  std::vector<double> trace;
  std::string err;
  Geometry geo{};
  // launch accounting
  int timing = 0;
  int64_t launches[RECON_K_COUNT] = {};
  double ms[RECON_K_COUNT] = {};
  double bytes[RECON_K_COUNT] = {};
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  // the instantiated iteration graph of the last device-driven recon_iterate(_from), relaunched
  // while every value it captured is unchanged (see GraphKey)
  struct GraphKey {
    uint32_t coef0_bits;
    const float* u0;
    int level, max_iter, d_is_k, generic, narrow, planes, tma, radix;
    uint64_t tol_bits;
    uint64_t epoch;
    bool operator==(const GraphKey& o) const {
      return coef0_bits == o.coef0_bits && u0 == o.u0 && level == o.level && max_iter == o.max_iter &&
             d_is_k == o.d_is_k && generic == o.generic && narrow == o.narrow && planes == o.planes && tma == o.tma &&
             radix == o.radix &&
             tol_bits == o.tol_bits &&
             epoch == o.epoch;
    }
  };
  struct GraphCache {
    bool valid = false;
    GraphKey key{};
    cudaGraph_t start = nullptr, whole = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t start_launches[RECON_K_COUNT] = {}, body_launches[RECON_K_COUNT] = {};
    double start_bytes[RECON_K_COUNT] = {}, body_bytes[RECON_K_COUNT] = {};
  } gcache;
  uint64_t epoch = 0;   // incremented whenever the per-reconstruction parameters change
};

#define RG_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) {                                     \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return RECON_ERR_CUDA;                                     \
    }                                                            \
  } while (0)

namespace {

// Run one kernel launch, counting it and, when timing is on, bracketing it with events.
template <class F>
cudaError_t timed(recon_handle* h, int kind, double alg_bytes, F&& launch) {
  h->launches[kind] += 1;
  h->bytes[kind] += alg_bytes;
  if (!h->timing) return launch();
  recon_handle::Pending p{kind, nullptr, nullptr};
  cudaError_t e;
  if ((e = cudaEventCreate(&p.a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&p.b)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(p.a, h->st)) != cudaSuccess) return e;
  if ((e = launch()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(p.b, h->st)) != cudaSuccess) return e;
  h->pending.push_back(p);
  return cudaSuccess;
}

cudaError_t drain_timing(recon_handle* h) {
  cudaError_t first = cudaSuccess;
  for (auto& p : h->pending) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e == cudaSuccess) h->ms[p.kind] += t;
    else if (first == cudaSuccess) first = e;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  h->pending.clear();
  return first;
}

int zkind(int mode) {
  switch (mode) {
    case Z_FWD: return RECON_K_ZFWD;
    case Z_INV: return RECON_K_ZINV;
    case Z_DELTA: return RECON_K_ZDELTA;
    case Z_PROJ: return RECON_K_ZPROJ;
    default: return RECON_K_ZFINAL;
  }
}

int skind(int mode, int axis) {
  switch (mode) {
    case S_DELTA: return RECON_K_KDELTA;
    case S_ITER: return RECON_K_KITER;
    default: return axis == AX_X ? (mode == S_FWD ? RECON_K_LINE_FWD : RECON_K_LINE_INV) : RECON_K_OTHER;
  }
}

Field field_at(char* base, const Layout& l) {
  Field f;
  f.M = reinterpret_cast<float2*>(base);
  f.Q = reinterpret_cast<float2*>(base + l.field_M);
  return f;
}

ZArgs zargs(recon_handle* h) {
  ZArgs a{};
  a.g = h->geo;
  a.tw = h->tw;
  a.tab = h->tabz;
  a.partials = h->partials;
  a.red = h->red;
  a.coef = 1.f;
  a.mask_frac = h->p.mask_frac;
  a.uniform = h->p.mean_density_mode == RECON_MEAN_UNIFORM;
  a.lognormal = h->p.lognormal;
  a.generic = h->kspace_generic;
  a.wf = h->W;
  return a;
}

SArgs sargs(recon_handle* h) {
  SArgs a{};
  a.g = h->geo;
  a.tab = h->tabs;
  a.partials = h->partials;
  a.red = h->red;
  a.dk = h->D;
  a.sbuf = h->S;
  a.inv_b = (float)(1.0 / h->p.b);
  a.beta = (float)(h->p.f / h->p.b);
  a.narrow = h->narrow_lines;
  a.generic = h->kspace_generic;
  a.lognormal = h->p.lognormal;
  a.tmaps = (h->tmaps_ok && h->kiter_tma) ? &h->tmaps : nullptr;
  a.wf = h->W;
  return a;
}

// Tensor maps of the fused source update's inputs (A in the third field, P_y in the second,
// delta(k), S) over the half grid M [kx][ky][kz < N/2], float2 elements copied as 8-byte words: boxes
// of 4 kz x 256 ky x 1 kx (a tile's y line is two boxes).  Needs the driver's encoder; without it the
// update loads its inputs directly.
bool encode_kiter_maps(recon_handle* h) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int n = h->n;
  const Field* fs[4] = {&h->V[2], &h->V[1], &h->D, &h->S};
  const cuuint64_t dims[3] = {(cuuint64_t)n / 2, (cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)(n / 2) * 8, (cuuint64_t)n * (n / 2) * 8};
  const cuuint32_t box[3] = {4, (cuuint32_t)(n / 2), 1};
  const cuuint32_t es[3] = {1, 1, 1};
  for (int q = 0; q < 4; ++q) {
    if (((uintptr_t)fs[q]->M & 255) != 0) return false;
    const CUresult r = encode(&h->tmaps.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)fs[q]->M, dims, strides, box, es,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

// Algorithmic bytes of one pass: every field it reads and writes, once.
double cfield(const recon_handle* h) { return (double)h->n * h->n * h->n * 4.0 + (double)h->n * h->n * 8.0; }
double rfield(const recon_handle* h) { return (double)h->n * h->n * h->n * 4.0; }

double zbytes(const recon_handle* h, int mode, int nc, const ZArgs& a) {
  // the register-fused path hands the z pass three fields (two in C form) and takes two back (psi^, Z^)
  const int nv = (h->mk->kspace_fused && !h->kspace_generic && nc == 3) ? 2 : nc;
  if (mode == Z_PROJ && a.cform) return 4.0 * cfield(h);
  if (mode == Z_DELTA) {
    const int nin = a.uniform ? 1 : 2;
    return nin * rfield(h) + cfield(h) + (a.delta_real ? rfield(h) : 0.0);
  }
  if (mode == Z_FINAL) return nc * (cfield(h) + rfield(h));
  if (mode == Z_RADIAL) return (a.cform ? 2 : nc) * cfield(h) + rfield(h);
  if (mode == Z_USTART || mode == Z_WARM) return rfield(h) + nv * cfield(h);
  return (nc + nv) * cfield(h);
}

double sbytes(const recon_handle* h, int mode, int nc, int axis, int cform) {
  // the register-fused path carries the x and z components of k-space vectors as one field
  const bool fused = h->mk->kspace_fused && !h->kspace_generic;
  if (mode == S_DELTA) return (fused ? 5.0 : 6.0) * cfield(h);   // delta in, delta(k), S, 2 or 3 Psi
  if (mode == S_ITER) return (fused ? 7.0 : 9.0) * cfield(h);    // 2 or 3 P + delta(k) + S in; 2 or 3 Psi + S out
  // paired x passes: inverse 2 fields in, 3 out (2 in C form); forward 2 in (the pair's shared one
  // read once), 2 out
  if (fused && axis == AX_X && nc == 3) return (mode == S_INV && !cform ? 5.0 : 4.0) * cfield(h);
  return 2.0 * nc * cfield(h);
}

recon_status run_z(recon_handle* h, int mode, int nc, const ZArgs& a, int* grid = nullptr) {
  const double part = a.ycount ? (double)a.ycount / h->n : 1.0;   // a batch of y-planes
  RG_CUDA(timed(h, zkind(mode), part * zbytes(h, mode, nc, a), [&] { return h->mk->zpass(mode, nc, a, h->st, grid); }));
  return RECON_OK;
}

recon_status run_s(recon_handle* h, int mode, int nc, int axis, const SArgs& a) {
  const double part = a.ycount ? (double)a.ycount / h->n : 1.0;
  RG_CUDA(timed(h, skind(mode, axis), part * sbytes(h, mode, nc, axis, a.cform), [&] { return h->mk->spass(mode, nc, axis, a, h->st); }));
  return RECON_OK;
}



recon_status finalize(recon_handle* h, int nblocks, int nq, int dst, int accumulate) {
  RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * nblocks * nq, [&] {
    return launch_finalize(h->partials, nblocks, nq, h->red, dst, accumulate, h->st, h->fin_bsum, h->fin_counter); }));
  return RECON_OK;
}

#define RG_TRY(x)                      \
  do {                                 \
    recon_status s_ = (x);             \
    if (s_ != RECON_OK) return s_;     \
  } while (0)

// Whether the x -> z -> x passes of an update run in batches of y-planes (register-fused path):
// the x passes transform lines at fixed (y, kz) and the z pass rows at fixed (x, y), so each batch
// of planes can go through all three before the next, and its fields stay in the L2 in between.
int plane_batch(const recon_handle* h) {
  return (h->plane_batch && h->mk->kspace_fused && !h->kspace_generic) ? h->plane_batch : 0;
}

// Whether the inverse x pass and the projection (or radial) pass exchange C = dx Psi_x + dy Psi_y
// and Psi_z (register-fused path) rather than the three components.
int cform(const recon_handle* h) {
  return (h->mk->kspace_fused && !h->kspace_generic && h->lay.wfield) ? 1 : 0;
}

// Inverse x, the projection pass and forward x over all y-planes, batch by batch.  za and the x
// arguments carry the device loop's flags when the passes run inside the iteration graph.
recon_status xzx_batched(recon_handle* h, int B, const ZArgs& za0, const int* skip_flag) {
  for (int y0 = 0; y0 < h->n; y0 += B) {
    SArgs xa = sargs(h);
    for (int q = 0; q < 3; ++q) xa.f[q] = h->V[q];
    xa.ybeg = y0;
    xa.ycount = B;
    xa.cform = cform(h);
    xa.loop_flag = skip_flag;
    RG_TRY(run_s(h, S_INV, 3, AX_X, xa));
    xa.loop_flag = nullptr;
    ZArgs za = za0;
    za.ybeg = y0;
    za.ycount = B;
    za.cform = xa.cform;
    RG_TRY(run_z(h, Z_PROJ, 3, za));
    xa.skip_flag = skip_flag;
    RG_TRY(run_s(h, S_FWD, 3, AX_X, xa));
  }
  return RECON_OK;
}

// plain X pass (one FFT along x per component) over nc fields.  The forward 3-D transform runs
// Z (r2c) -> X -> Y, the inverse Y -> X -> Z; the Y passes carry the k-space work.
recon_status xpass(recon_handle* h, int mode, int nc, const Field* f, int cf = 0, const int* flag = nullptr) {
  SArgs a = sargs(h);
  for (int q = 0; q < nc; ++q) a.f[q] = f[q];
  a.cform = cf;
  a.loop_flag = flag;
  return run_s(h, mode, nc, AX_X, a);
}

size_t elem_size(int dtype) { return dtype == RECON_F64 ? 8 : 4; }

recon_status check_catalog(const recon_catalog* c) {
  if (!c) return RECON_ERR_INVALID_ARG;
  if (c->n < 0) return RECON_ERR_INVALID_ARG;
  if (c->n > 0 && !c->pos) return RECON_ERR_INVALID_ARG;
  if (c->dtype != RECON_F64 && c->dtype != RECON_F32) return RECON_ERR_INVALID_ARG;
  return RECON_OK;
}

// Deposit one catalogue into rho; the weight sum goes to red[slot].  Particles go through in chunks
// (staged through the host buffer when the catalogue is in host memory), either directly (global
// atomics per particle) or brick-sorted into the shared-memory binned deposit.
// The device-side address of page-locked host memory (null for other host memory).
const void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

recon_status deposit_one(recon_handle* h, const recon_catalog* c, float* rho, int slot) {
  const size_t es = elem_size(c->dtype);
  // nearest-grid-point binning has no brick-sorted form: it always takes the direct kernel
  const int path = h->assign ? RECON_PATH_DIRECT : h->deposit_path;
  if (!c->on_device && c->n > 0 && path == RECON_PATH_DIRECT) {
    // page-locked host catalogue: the direct deposit reads it where it is, in one launch
    const void* dpos = mapped_host(c->pos);
    const float* dw = c->w ? static_cast<const float*>(mapped_host(c->w)) : nullptr;
    if (dpos && (!c->w || dw)) {
      RG_CUDA(timed(h, RECON_K_DEPOSIT, (double)c->n * (3 * es + (c->w ? 4 : 0)), [&] {
        return launch_deposit(dpos, c->dtype, dw, c->n, h->n, h->L, rho, h->partials, kDepositBlocks, h->st,
                              h->assign); }));
      RG_TRY(finalize(h, kDepositBlocks, 1, slot, 0));
      return RECON_OK;
    }
  }
  if (path == RECON_PATH_SORTED && c->n > 0 && c->n <= h->bb.chunk) {
    // the whole catalogue in one sort (page-locked host memory is read in place); the sort
    // buffers then hold its brick order for a later shift of the same catalogue
    const void* dpos = c->on_device ? c->pos : mapped_host(c->pos);
    const float* dw = c->w ? (c->on_device ? c->w : static_cast<const float*>(mapped_host(c->w))) : nullptr;
    if (dpos && (!c->w || dw)) {
      h->memo.valid = 0;
      RG_CUDA(timed(h, RECON_K_SORT, (double)c->n * (6 * es + (c->w ? 4 : 0) + 44),
                    [&] { return brick_sort(h->bb, dpos, c->dtype, dw, c->n, h->st); }));
      RG_CUDA(timed(h, RECON_K_DEPOSIT, (double)c->n * 16, [&] { return brick_deposit(h->bb, rho, h->partials, h->st); }));
      RG_TRY(finalize(h, brick_grid(), 1, slot, 0));
      h->memo = {1, c->pos, c->n, c->dtype, c->on_device};
      return RECON_OK;
    }
  }
  const long long chunk = c->on_device ? h->bb.chunk : (kStageParticles < h->bb.chunk ? kStageParticles : h->bb.chunk);
  char* spos = h->stage;
  float* sw = reinterpret_cast<float*>(h->stage + kStageParticles * 24);
  if (c->n == 0) RG_CUDA(cudaMemsetAsync(h->red + slot, 0, sizeof(double), h->st));
  if (path == RECON_PATH_SORTED) h->memo.valid = 0;
  for (long long p0 = 0; p0 < c->n; p0 += chunk) {
    const long long m = (c->n - p0 < chunk) ? c->n - p0 : chunk;
    const void* pin = (const char*)c->pos + (size_t)p0 * 3 * es;
    const float* win = c->w ? c->w + p0 : nullptr;
    if (!c->on_device) {
      RG_CUDA(cudaMemcpyAsync(spos, pin, (size_t)m * 3 * es, cudaMemcpyHostToDevice, h->st));
      pin = spos;
      if (c->w) {
        RG_CUDA(cudaMemcpyAsync(sw, c->w + p0, (size_t)m * sizeof(float), cudaMemcpyHostToDevice, h->st));
        win = sw;
      }
    }
    if (path == RECON_PATH_SORTED) {
      RG_CUDA(timed(h, RECON_K_SORT, (double)m * (6 * es + (c->w ? 4 : 0) + 28),
                    [&] { return brick_sort(h->bb, pin, c->dtype, win, m, h->st); }));
      RG_CUDA(timed(h, RECON_K_DEPOSIT, (double)m * 16, [&] { return brick_deposit(h->bb, rho, h->partials, h->st); }));
      RG_TRY(finalize(h, brick_grid(), 1, slot, p0 > 0));
    } else {
      RG_CUDA(timed(h, RECON_K_DEPOSIT, (double)m * (3 * es + (c->w ? 4 : 0)), [&] {
        return launch_deposit(pin, c->dtype, win, m, h->n, h->L, rho, h->partials, kDepositBlocks, h->st,
                              h->assign); }));
      RG_TRY(finalize(h, kDepositBlocks, 1, slot, p0 > 0));
    }
  }
  return RECON_OK;
}

// Copy a half-grid field (M, Q) into the standard [kx][ky][kz = 0..N/2] layout (or back).
recon_status export_half(recon_handle* h, const Field& f, float* out) {
  const int n = h->n;
  const size_t H = n / 2;
  RG_CUDA(cudaMemcpy2DAsync(out, (H + 1) * sizeof(float2), f.M, H * sizeof(float2), H * sizeof(float2),
                            (size_t)n * n, cudaMemcpyDefault, h->st));
  RG_CUDA(cudaMemcpy2DAsync(reinterpret_cast<float2*>(out) + H, (H + 1) * sizeof(float2), f.Q, sizeof(float2),
                            sizeof(float2), (size_t)n * n, cudaMemcpyDefault, h->st));
  return RECON_OK;
}

recon_status import_half(recon_handle* h, const float* in, const Field& f) {
  const int n = h->n;
  const size_t H = n / 2;
  RG_CUDA(cudaMemcpy2DAsync(f.M, H * sizeof(float2), in, (H + 1) * sizeof(float2), H * sizeof(float2),
                            (size_t)n * n, cudaMemcpyDefault, h->st));
  RG_CUDA(cudaMemcpy2DAsync(f.Q, sizeof(float2), reinterpret_cast<const float2*>(in) + H, (H + 1) * sizeof(float2),
                            sizeof(float2), (size_t)n * n, cudaMemcpyDefault, h->st));
  return RECON_OK;
}

double start_coefficient(int start, double beta) {
  if (start == RECON_START_APPROX1) return beta / (1.0 + beta);
  if (start == RECON_START_FFTA) return 3.0 * beta / (7.0 + 3.0 * beta);
  return 0.0;
}

}  // namespace

namespace rg {

// Host tables of one parameter set: node offsets from the observer (3 N floats; x then y then z)
// and the Gaussian smoothing kernel as a periodic convolution per axis,
// g[t] = (1/N) sum_m exp(-k_m^2 R^2/2) cos(2 pi m t / N); taps beyond the last |g[t]| > 1e-9 g[0]
// are dropped, and a kernel that has not decayed by then is used over the whole period.
void config_tables(int n, const recon_params* p, std::vector<float>& taps, int* t0, int* ntap,
                   std::vector<float>& off) {
  const double L = p->box[0];
  off.assign(3 * n, 0.f);
  const double H = L / n;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n; ++i) off[a * n + i] = (float)((double)i * H - p->observer[a]);
  std::vector<double> gk(n);
  for (int t = 0; t < n; ++t) {
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
      const int mm = (m <= n / 2) ? m : m - n;
      const double k = 2.0 * M_PI * mm / L;
      acc += std::exp(-0.5 * k * k * p->smooth_R * p->smooth_R) * std::cos(2.0 * M_PI * (double)m * t / n);
    }
    gk[t] = acc / n;
  }
  int K = 0;
  for (int t = 1; t <= n / 2; ++t)
    if (std::fabs(gk[t]) > 1e-9 * std::fabs(gk[0])) K = t;
  if (2 * K + 1 >= n) {
    *t0 = -n / 2;
    *ntap = n;
  } else {
    *t0 = -K;
    *ntap = 2 * K + 1;
  }
  taps.assign(*ntap, 0.f);
  for (int j = 0; j < *ntap; ++j) taps[j] = (float)gk[((*t0 + j) % n + n) % n];
}

}  // namespace rg

namespace {

// Point the handle at a parameter set whose tables already sit in device memory (taps_dev holds
// ntap floats, off_dev 3 N floats), without touching the device; resets the call sequence.
void apply_config(recon_handle* h, const recon_params* p, const float* taps_dev, int t0, int ntap,
                  const float* off_dev) {
  h->memo.valid = 0;
  h->p = *p;
  h->L = p->box[0];
  h->bb.scale = (double)h->n / h->L;
  h->t0 = t0;
  h->ntap = ntap;
  h->cur_taps = taps_dev;
  h->cur_off = off_dev;
  const int n = h->n;
  Geometry& g = h->geo;
  g.n = n;
  g.kf = (float)(2.0 * M_PI / h->L);
  g.inv_n3 = (float)(1.0 / ((double)n * n * n));
  g.los_mode = p->los_mode;
  if (p->los_mode == RECON_LOS_FIXED) {
    const double q = std::sqrt(p->observer[0] * p->observer[0] + p->observer[1] * p->observer[1] +
                               p->observer[2] * p->observer[2]);
    g.los = make_float3((float)(p->observer[0] / q), (float)(p->observer[1] / q), (float)(p->observer[2] / q));
  } else {
    g.los = make_float3(0.f, 0.f, 0.f);
  }
  g.off = off_dev;
  ++h->epoch;   // kernel arguments captured in a cached iteration graph are now stale
  h->state = ST_CREATED;
  h->warm_level = -1;
  h->d_is_k = 0;
  h->delta_real_valid = 0;
}

// Per-reconstruction parameters that do not change the mesh: box, bias, growth rate, smoothing
// length, line of sight, mask and density options.  Uploads the node offsets from the observer and
// the smoothing taps into the handle's own tables, and resets the call sequence.
recon_status configure(recon_handle* h, const recon_params* p) {
  std::vector<float> taps, off;
  int t0 = 0, ntap = 1;
  config_tables(h->n, p, taps, &t0, &ntap, off);
  RG_CUDA(cudaMemcpyAsync(h->taps, taps.data(), ntap * sizeof(float), cudaMemcpyHostToDevice, h->st));
  RG_CUDA(cudaMemcpyAsync(h->off, off.data(), 3 * h->n * sizeof(float), cudaMemcpyHostToDevice, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));   // the host vectors go out of scope
  apply_config(h, p, h->taps, t0, ntap, h->off);
  return RECON_OK;
}

}  // namespace

extern "C" {

const char* recon_status_str(recon_status s) {
  switch (s) {
    case RECON_OK: return "ok";
    case RECON_ERR_INVALID_ARG: return "invalid argument";
    case RECON_ERR_OOM: return "out of device memory or workspace too small";
    case RECON_ERR_CUDA: return "CUDA error";
    case RECON_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case RECON_ERR_NONFINITE: return "non-finite value in the convergence norms";
    case RECON_ERR_STATE: return "call out of order";
    case RECON_ERR_TIMEOUT: return "bounded device wait timed out";
    case RECON_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* recon_last_error(recon_handle* h) { return h ? h->err.c_str() : ""; }

recon_status recon_workspace_bytes(const recon_params* p, size_t* bytes) {
  if (!valid_params(p) || !bytes) return RECON_ERR_INVALID_ARG;
  *bytes = layout_for(p->nmesh[0]).total;
  return RECON_OK;
}

recon_status recon_create(const recon_params* p, void* stream, void* workspace, size_t workspace_bytes,
                          recon_handle** out) {
  if (!out || !valid_params(p)) return RECON_ERR_INVALID_ARG;
  *out = nullptr;
  recon_handle* h = new recon_handle();
  h->p = *p;
  h->n = p->nmesh[0];
  h->L = p->box[0];
  h->st = (cudaStream_t)stream;
  h->mk = mesh_kernels(h->n);
  h->lay = layout_for(h->n);
  cudaGetDevice(&h->device);
  if (workspace) {
    if (workspace_bytes < h->lay.total || ((uintptr_t)workspace & 255)) {
      delete h;
      return ((uintptr_t)workspace & 255) ? RECON_ERR_INVALID_ARG : RECON_ERR_OOM;
    }
    h->ws = (char*)workspace;
    h->ws_bytes = workspace_bytes;
  } else {
    if (cudaMalloc(&h->ws, h->lay.total) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return RECON_ERR_OOM;
    }
    h->own_ws = true;
    h->ws_bytes = h->lay.total;
  }
  char* b = h->ws;
  for (int q = 0; q < 3; ++q, b += h->lay.field) h->V[q] = field_at(b, h->lay);
  h->D = field_at(b, h->lay);
  b += h->lay.field;
  h->S = field_at(b, h->lay);
  b += h->lay.field;
  if (h->lay.wfield) {
    h->W = field_at(b, h->lay);
    b += h->lay.wfield;
  }
  h->tw = (float2*)b;
  b += h->lay.tw;
  h->tabs = (float2*)b;
  b += h->lay.tabs;
  h->tabz = (float2*)b;
  b += h->lay.tabz;
  h->off = (float*)b;
  b += h->lay.off;
  h->taps = (float*)b;
  b += h->lay.taps;
  h->red = (double*)b;
  h->loop = reinterpret_cast<LoopState*>(h->red + 64);
  h->fin_bsum = reinterpret_cast<double*>(h->loop + 1);
  h->fin_counter = reinterpret_cast<unsigned int*>(h->fin_bsum + kFinalizeBlocks * 4);
  b += h->lay.red;
  h->partials = (double*)b;
  b += h->lay.partials;
  h->stage = b;
  b += h->lay.stage;
  h->bb = brick_buffers(b, h->n, h->L);
  b += h->lay.bricks;
  h->ucoarse = (float*)b;

  // twiddles exp(-2 pi i m / N), computed in float64, and the stage tables built from them
  const int n = h->n;
  std::vector<float2> tw(n);
  for (int m = 0; m < n; ++m) {
    const double ang = -2.0 * M_PI * (double)m / (double)n;
    tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  recon_status rs = RECON_OK;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->tw, tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice, h->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->red, 0, h->lay.red, h->st)) != cudaSuccess ||
      (e = h->mk->build_tables(h->tw, h->tabs, h->tabz, h->st)) != cudaSuccess) {
    h->err = cudaGetErrorString(e);
    rs = RECON_ERR_CUDA;
  }
  if (rs == RECON_OK) rs = configure(h, p);
  if (rs == RECON_OK && h->mk->kspace_fused) h->tmaps_ok = encode_kiter_maps(h);
  if (rs != RECON_OK) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return rs;
  }
  *out = h;
  return RECON_OK;
}

recon_status recon_reconfigure(recon_handle* h, const recon_params* p) {
  if (!h || !valid_params(p) || p->nmesh[0] != h->n) return RECON_ERR_INVALID_ARG;
  return configure(h, p);
}

recon_status recon_set_timing(recon_handle* h, int enable) {
  if (!h) return RECON_ERR_INVALID_ARG;
  h->timing = enable ? 1 : 0;
  return RECON_OK;
}

recon_status recon_get_timing(recon_handle* h, int kind, double* total_ms, int64_t* launches,
                              double* alg_bytes) {
  if (!h || kind < 0 || kind >= RECON_K_COUNT) return RECON_ERR_INVALID_ARG;
  RG_CUDA(drain_timing(h));
  if (total_ms) *total_ms = h->ms[kind];
  if (launches) *launches = h->launches[kind];
  if (alg_bytes) *alg_bytes = h->bytes[kind];
  return RECON_OK;
}

recon_status recon_reset_timing(recon_handle* h) {
  if (!h) return RECON_ERR_INVALID_ARG;
  RG_CUDA(drain_timing(h));
  for (int k = 0; k < RECON_K_COUNT; ++k) {
    h->ms[k] = 0.0;
    h->bytes[k] = 0.0;
    h->launches[k] = 0;
  }
  return RECON_OK;
}

recon_status set_plane_batch(recon_handle* h, int value);
recon_status set_radix_order(recon_handle* h, int value);

recon_status recon_set_option(recon_handle* h, int option, int value) {
  if (!h) return RECON_ERR_INVALID_ARG;
  if (option == RECON_OPT_PLANE_BATCH) return set_plane_batch(h, value);
  if (value != 0 && value != 1) return RECON_ERR_INVALID_ARG;
  if (option == RECON_OPT_FFT_RADIX) return set_radix_order(h, value);
  if (option == RECON_OPT_DEPOSIT_PATH) h->deposit_path = value;
  else if (option == RECON_OPT_SHIFT_PATH) h->shift_path = value;
  else if (option == RECON_OPT_GRAPH) h->use_graph = value;
  else if (option == RECON_OPT_LINE_TILE) h->narrow_lines = value;
  else if (option == RECON_OPT_KSPACE_GENERIC) h->kspace_generic = value ? 1 : 0;
  else if (option == RECON_OPT_REUSE_SORT) h->reuse_sort = value ? 1 : 0;
  else if (option == RECON_OPT_ASSIGN) h->assign = value;
  else if (option == RECON_OPT_KITER_TMA) h->kiter_tma = value;
  else return RECON_ERR_INVALID_ARG;
  return RECON_OK;
}

// Switch the FFT plans to another radix order: that order's kernels, and its stage tables rebuilt
// (in place: the layout has room for either order) on the handle's stream.
recon_status set_radix_order(recon_handle* h, int value) {
  const MeshKernels* mk = mesh_kernels_order(h->n, value);
  if (!mk) return RECON_ERR_UNSUPPORTED;
  if (value == h->radix_order) return RECON_OK;
  RG_CUDA(mk->build_tables(h->tw, h->tabs, h->tabz, h->st));
  h->mk = mk;
  h->radix_order = value;
  return RECON_OK;
}

recon_status set_plane_batch(recon_handle* h, int value) {
  if (value != 0 && value != 16 && value != 32 && value != 64) return RECON_ERR_INVALID_ARG;
  h->plane_batch = value;
  return RECON_OK;
}

namespace {
void drop_graph(recon_handle* h);   // releases the cached iteration graph (defined with it below)
}  // namespace

recon_status recon_destroy(recon_handle* h) {
  if (!h) return RECON_OK;
  drain_timing(h);
  drop_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->copy_st) {
    cudaStreamSynchronize(h->copy_st);
    cudaStreamDestroy(h->copy_st);
    for (int b = 0; b < 2; ++b) {
      cudaEventDestroy(h->ev_in[b]);
      cudaEventDestroy(h->ev_out[b]);
      cudaEventDestroy(h->ev_free[b]);
    }
  }
  if (h->own_ws && h->ws) {
    cudaStreamSynchronize(h->st);
    cudaFree(h->ws);
  }
  delete h;
  return RECON_OK;
}

recon_status recon_deposit(recon_handle* h, const recon_catalog* gal, const recon_catalog* ran) {
  if (!h) return RECON_ERR_INVALID_ARG;
  RG_TRY(check_catalog(gal));
  const bool uniform = h->p.mean_density_mode == RECON_MEAN_UNIFORM;
  if (gal->n == 0) return RECON_ERR_INVALID_ARG;
  if (!uniform) {
    if (!ran) return RECON_ERR_INVALID_ARG;
    RG_TRY(check_catalog(ran));
    if (ran->n == 0) return RECON_ERR_INVALID_ARG;
  }
  const size_t bytes = (size_t)h->n * h->n * h->n * sizeof(float);
  h->memo.valid = 0;
  RG_CUDA(cudaMemsetAsync(h->red, 0, h->lay.red, h->st));
  RG_CUDA(cudaMemsetAsync(h->V[0].M, 0, bytes, h->st));
  RG_TRY(deposit_one(h, gal, reinterpret_cast<float*>(h->V[0].M), RED_SUM_WG));
  if (!uniform) {
    RG_CUDA(cudaMemsetAsync(h->V[1].M, 0, bytes, h->st));
    RG_TRY(deposit_one(h, ran, reinterpret_cast<float*>(h->V[1].M), RED_SUM_WR));
  }
  // host catalogues are borrowed for the call only: they are read before it returns
  if (!gal->on_device || (ran && ran->n > 0 && !ran->on_device)) RG_CUDA(cudaStreamSynchronize(h->st));
  h->state = ST_DEPOSITED;
  h->delta_real_valid = 0;
  h->warm_level = -1;
  h->d_is_k = 0;
  return RECON_OK;
}

recon_status recon_smooth(recon_handle* h) {
  if (!h) return RECON_ERR_INVALID_ARG;
  if (h->state != ST_DEPOSITED) return RECON_ERR_STATE;
  const bool uniform = h->p.mean_density_mode == RECON_MEAN_UNIFORM;
  const int nf = uniform ? 1 : 2;
  ConvArgs c{};
  c.f[0] = reinterpret_cast<float*>(h->V[0].M);
  c.f[1] = reinterpret_cast<float*>(h->V[1].M);
  c.nf = nf;
  c.n = h->n;
  c.taps = h->cur_taps;
  c.ntap = h->ntap;
  c.t0 = h->t0;
  c.partials = h->partials;
  // x factor of the Gaussian; counts the nodes that received random mass (mask threshold)
  c.axis = 0;
  c.count = !uniform;
  RG_CUDA(timed(h, RECON_K_CONV, 2.0 * nf * rfield(h), [&] { return launch_conv(c, h->st); }));
  if (!uniform) RG_TRY(finalize(h, conv_blocks(h->n), 2, RED_SUM_RPOS, 0));
  // y factor
  c.axis = 1;
  c.count = 0;
  RG_CUDA(timed(h, RECON_K_CONV, 2.0 * nf * rfield(h), [&] { return launch_conv(c, h->st); }));
  // z factor, delta (mask, lognormal) and its r2c along z
  {
    ZArgs a = zargs(h);
    a.f[0] = h->V[0];
    a.f[1] = h->V[1];
    a.dout = h->D;
    a.delta_real = reinterpret_cast<float*>(h->V[2].M);
    a.taps = h->cur_taps;
    a.ntap = h->ntap;
    a.t0 = h->t0;
    int zg = 0;
    RG_TRY(run_z(h, Z_DELTA, 2, a, &zg));
    RG_TRY(finalize(h, zg, 2, RED_SUM_LOG, 0));
  }
  RG_TRY(xpass(h, S_FWD, 1, &h->D));
  h->state = ST_SMOOTHED;
  h->d_is_k = 0;
  h->delta_real_valid = 1;
  return RECON_OK;
}

namespace {

// Start of the iteration (Sec. 5.2): delta(k), S_-1 = delta/b, Psi_s = Z[delta/b] along y, back to
// configuration space, P_0 = (1 - c)(Psi_s.r) r, forward along z and x.
recon_status iterate_start(recon_handle* h, float coef0) {
  {
    SArgs a = sargs(h);
    for (int q = 0; q < 3; ++q) a.f[q] = h->V[q];
    a.d_is_k = h->d_is_k;
    RG_TRY(run_s(h, S_DELTA, 1, AX_Y, a));
  }
  ZArgs za = zargs(h);
  for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
  za.coef = coef0;
  if (const int B = plane_batch(h)) return xzx_batched(h, B, za, nullptr);
  za.cform = cform(h);
  RG_TRY(xpass(h, S_INV, 3, h->V, za.cform));
  RG_TRY(run_z(h, Z_PROJ, 3, za));
  RG_TRY(xpass(h, S_FWD, 3, h->V));
  return RECON_OK;
}

// One update of Eq. iterative inside the device-driven loop: S_n, norms, Psi_n+1 = Z[S_n] along y;
// the decide kernel records rel and ends the loop on convergence, after which the Z pass writes
// the real Psi and the forward x pass is skipped.
recon_status iterate_body(recon_handle* h, cudaGraphConditionalHandle cond) {
  SArgs ia = sargs(h);
  for (int q = 0; q < 3; ++q) ia.f[q] = h->V[q];
  RG_TRY(run_s(h, S_ITER, 3, AX_Y, ia));
  RG_TRY(finalize(h, h->mk->s_blocks, 2, RED_NORM_D2, 0));
  RG_CUDA(timed(h, RECON_K_OTHER, 0.0, [&] { return launch_loop_decide(h->loop, h->red, cond, h->st); }));
  ZArgs za = zargs(h);
  for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
  za.loop_flag = &h->loop->flag;
  if (const int B = plane_batch(h)) return xzx_batched(h, B, za, &h->loop->flag);
  // C form unless the decide kernel has just ended the loop (then the Z pass writes the real Psi)
  za.cform = cform(h);
  RG_TRY(xpass(h, S_INV, 3, h->V, za.cform, &h->loop->flag));
  RG_TRY(run_z(h, Z_PROJ, 3, za));
  SArgs fa = sargs(h);
  for (int q = 0; q < 3; ++q) fa.f[q] = h->V[q];
  fa.skip_flag = &h->loop->flag;
  RG_TRY(run_s(h, S_FWD, 3, AX_X, fa));
  return RECON_OK;
}

// How the iteration starts: the analytic start (coefficient 1 - c), a supplied radial displacement
// on the mesh, or the warm start prepared by recon_start_features plus a coarse correction.
struct StartSpec {
  float coef0 = 1.f;
  const float* u0 = nullptr;
  int level = 0;
};
recon_status run_start(recon_handle* h, const StartSpec& sp);

void drop_graph(recon_handle* h) {
  auto& c = h->gcache;
  if (c.exec) cudaGraphExecDestroy(c.exec);
  if (c.whole) cudaGraphDestroy(c.whole);
  if (c.start) cudaGraphDestroy(c.start);
  c = recon_handle::GraphCache{};
}

// The whole iteration as one CUDA graph: the start sequence, then a conditional WHILE node whose
// body is one update.  One launch, one host synchronisation at the end.  The instantiated graph is
// kept on the handle and relaunched by later calls whose captured values (start coefficient or
// supplied displacement, level, tol, max_iter, options, parameters) are the same; anything else
// rebuilds it.
recon_status build_graph(recon_handle* h, const StartSpec& sp, double tol, int max_iter) {
  drop_graph(h);
  auto& c = h->gcache;
  if (!h->cap_stream) RG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const cudaStream_t user = h->st;
  int64_t l0[RECON_K_COUNT], l1[RECON_K_COUNT];
  double b0[RECON_K_COUNT], b1[RECON_K_COUNT];
  for (int k = 0; k < RECON_K_COUNT; ++k) {
    l0[k] = h->launches[k];
    b0[k] = h->bytes[k];
  }
  recon_status rs = RECON_OK;
  h->st = h->cap_stream;
  do {
    cudaError_t e;
    if ((e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    rs = [&]() -> recon_status {
      RG_CUDA(launch_loop_init(h->loop, tol, max_iter, h->st));
      return run_start(h, sp);
    }();
    e = cudaStreamEndCapture(h->st, &c.start);
    if (rs != RECON_OK) break;
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    for (int k = 0; k < RECON_K_COUNT; ++k) {
      l1[k] = h->launches[k];
      b1[k] = h->bytes[k];
    }
    if ((e = cudaGraphCreate(&c.whole, 0)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraphNode_t child = nullptr, cnode = nullptr;
    if ((e = cudaGraphAddChildGraphNode(&child, c.whole, nullptr, 0, c.start)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, c.whole, 1, cudaGraphCondAssignDefault)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if ((e = cudaGraphAddNode(&cnode, c.whole, &child, nullptr, 1, &np)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    rs = iterate_body(h, cond);
    cudaGraph_t body_out = nullptr;
    e = cudaStreamEndCapture(h->st, &body_out);
    if (rs != RECON_OK) break;
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    if ((e = cudaGraphInstantiate(&c.exec, c.whole, 0)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
  } while (0);
  h->st = user;
  // capture recorded the launches once; they are counted per execution instead
  for (int k = 0; k < RECON_K_COUNT; ++k) {
    c.start_launches[k] = l1[k] - l0[k];
    c.start_bytes[k] = b1[k] - b0[k];
    c.body_launches[k] = h->launches[k] - l1[k];
    c.body_bytes[k] = h->bytes[k] - b1[k];
    h->launches[k] = l0[k];
    h->bytes[k] = b0[k];
  }
  if (rs != RECON_OK) {
    drop_graph(h);
    return rs;
  }
  c.valid = true;
  return RECON_OK;
}

recon_status iterate_graph(recon_handle* h, const StartSpec& sp, double tol, int max_iter, int* it_out,
                           double* rel_out, int* flag_out) {
  recon_handle::GraphKey key{};
  std::memcpy(&key.coef0_bits, &sp.coef0, sizeof(float));
  std::memcpy(&key.tol_bits, &tol, sizeof(double));
  key.u0 = sp.u0;
  key.level = sp.level;
  key.max_iter = max_iter;
  key.d_is_k = h->d_is_k;
  key.generic = h->kspace_generic;
  key.narrow = h->narrow_lines;
  key.planes = h->plane_batch;
  key.tma = h->kiter_tma;
  key.radix = h->radix_order;
  key.epoch = h->epoch;
  if (!(h->gcache.valid && h->gcache.key == key)) {
    RG_TRY(build_graph(h, sp, tol, max_iter));
    h->gcache.key = key;
  }
  RG_CUDA(cudaGraphLaunch(h->gcache.exec, h->st));
  int hdr[2];
  RG_CUDA(cudaMemcpyAsync(hdr, h->loop, sizeof(hdr), cudaMemcpyDeviceToHost, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));
  const int it = hdr[1];
  h->trace.assign(it < kMaxTrace ? it : kMaxTrace, 0.0);
  if (!h->trace.empty())
    RG_CUDA(cudaMemcpy(h->trace.data(), h->loop->trace, h->trace.size() * sizeof(double), cudaMemcpyDeviceToHost));
  // the start ran once and the body it times (its last pass skipped the forward x transforms)
  for (int k = 0; k < RECON_K_COUNT; ++k) {
    h->launches[k] += h->gcache.start_launches[k] + h->gcache.body_launches[k] * it;
    h->bytes[k] += h->gcache.start_bytes[k] + h->gcache.body_bytes[k] * it;
  }
  *it_out = it;
  *rel_out = h->trace.empty() ? 0.0 : h->trace.back();
  *flag_out = hdr[0];
  return RECON_OK;
}

}  // namespace

namespace {

// Start sequence for a supplied radial displacement u0 (device, N^3): delta(k) and S_-1 along y,
// then P_0 = u0 r transformed along z and x.
recon_status iterate_start_from(recon_handle* h, const float* u0) {
  {
    SArgs a = sargs(h);
    for (int q = 0; q < 3; ++q) a.f[q] = h->V[q];
    a.d_is_k = h->d_is_k;
    RG_TRY(run_s(h, S_DELTA, 1, AX_Y, a));
  }
  ZArgs za = zargs(h);
  for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
  za.u_in = u0;
  RG_TRY(run_z(h, Z_USTART, 3, za));
  RG_TRY(xpass(h, S_FWD, 3, h->V));
  return RECON_OK;
}

// Warm start: recon_start_features left delta(k), S_-1 and the start's radial displacement u_s
// (real, in the first vector field); P_0 = (u_s + up(u0 - mean(u_s))) r transformed along z and x.
recon_status iterate_start_warm(recon_handle* h, const float* u0, int level) {
  ZArgs za = zargs(h);
  for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
  za.u_in = reinterpret_cast<const float*>(h->V[0].M);
  za.corr = u0;
  za.ucoarse = h->ucoarse;
  za.clevel = level;
  RG_TRY(run_z(h, Z_WARM, 3, za));
  RG_TRY(xpass(h, S_FWD, 3, h->V));
  return RECON_OK;
}

recon_status run_start(recon_handle* h, const StartSpec& sp) {
  if (!sp.u0) return iterate_start(h, sp.coef0);
  if (sp.level == 0) return iterate_start_from(h, sp.u0);
  return iterate_start_warm(h, sp.u0, sp.level);
}

// The loop of Sec. 5.1 after a start: device-driven (one CUDA graph) or host-driven.
recon_status iterate_core(recon_handle* h, const StartSpec& sp, double tol, int max_iter, int* n_iter,
                          double* rel_change) {
  h->trace.clear();
  h->delta_real_valid = 0;
  h->warm_level = -1;
  double rel = 0.0;
  int it = 0;
  recon_status result = RECON_OK;
  if (h->use_graph && !h->timing && max_iter <= kMaxTrace) {
    int flag = 0;
    RG_TRY(iterate_graph(h, sp, tol, max_iter, &it, &rel, &flag));
    h->d_is_k = 1;
    if (flag == 2) {
      h->state = ST_SMOOTHED;
      result = RECON_ERR_NONFINITE;
    }
  } else {
    RG_TRY(run_start(h, sp));
    h->d_is_k = 1;
    ZArgs za = zargs(h);
    for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
    SArgs ia = sargs(h);
    for (int q = 0; q < 3; ++q) ia.f[q] = h->V[q];
    double host_norm[2] = {0, 0};
    while (true) {
      RG_TRY(run_s(h, S_ITER, 3, AX_Y, ia));
      RG_TRY(finalize(h, h->mk->s_blocks, 2, RED_NORM_D2, 0));
      RG_CUDA(cudaMemcpyAsync(host_norm, h->red + RED_NORM_D2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      cudaEvent_t ev;
      RG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      RG_CUDA(cudaEventRecord(ev, h->st));
      const int B = plane_batch(h);
      // the inverse waits for the decision: after the last update it writes the three components
      const int cf = cform(h);
      if (!B && !cf) RG_TRY(xpass(h, S_INV, 3, h->V));
      cudaError_t es = cudaEventSynchronize(ev);
      cudaEventDestroy(ev);
      RG_CUDA(es);
      ++it;
      if (!std::isfinite(host_norm[0]) || !std::isfinite(host_norm[1])) {
        h->state = ST_SMOOTHED;
        result = RECON_ERR_NONFINITE;
        break;
      }
      rel = host_norm[1] > 0 ? std::sqrt(host_norm[0] / host_norm[1]) : 0.0;
      h->trace.push_back(rel);
      const bool done = (it >= 2 && rel < tol) || it >= max_iter;
      if (done) {
        if (B || cf) RG_TRY(xpass(h, S_INV, 3, h->V));
        RG_TRY(run_z(h, Z_FINAL, 3, za));
        break;
      }
      if (B) {
        RG_TRY(xzx_batched(h, B, za, nullptr));
        continue;
      }
      if (cf) RG_TRY(xpass(h, S_INV, 3, h->V, cf));
      ZArgs zc = za;
      zc.cform = cf;
      RG_TRY(run_z(h, Z_PROJ, 3, zc));
      RG_TRY(xpass(h, S_FWD, 3, h->V));
    }
  }
  if (result == RECON_OK) {
    h->state = ST_ITERATED;
    if (tol > 0 && rel >= tol) result = RECON_ERR_NOT_CONVERGED;
  }
  if (n_iter) *n_iter = it;
  if (rel_change) *rel_change = rel;
  return result;
}

}  // namespace

recon_status recon_start_coefficient(int start, double beta, double* c) {
  if (!c || start < RECON_START_PLAIN || start > RECON_START_FFTA || !std::isfinite(beta) || beta < 0)
    return RECON_ERR_INVALID_ARG;
  *c = start_coefficient(start, beta);
  return RECON_OK;
}

recon_status recon_iterate(recon_handle* h, int start, double tol, int max_iter, int* n_iter, double* rel_change) {
  if (!h) return RECON_ERR_INVALID_ARG;
  if (h->state < ST_SMOOTHED) return RECON_ERR_STATE;
  if (max_iter < 1 || !(tol >= 0) || start < RECON_START_PLAIN || start > RECON_START_FFTA)
    return RECON_ERR_INVALID_ARG;
  const double beta = h->p.f / h->p.b;
  StartSpec sp;
  sp.coef0 = (float)(1.0 - start_coefficient(start, beta));
  return iterate_core(h, sp, tol, max_iter, n_iter, rel_change);
}

recon_status recon_iterate_from(recon_handle* h, const float* u0, int level, double tol, int max_iter, int* n_iter,
                                double* rel_change) {
  if (!h || !u0 || level < 0 || level > 2) return RECON_ERR_INVALID_ARG;
  if (h->state < ST_SMOOTHED) return RECON_ERR_STATE;
  if (max_iter < 1 || !(tol >= 0)) return RECON_ERR_INVALID_ARG;
  if (level > 0 && h->warm_level != level) return RECON_ERR_STATE;
  StartSpec sp;
  sp.u0 = u0;
  sp.level = level;
  return iterate_core(h, sp, tol, max_iter, n_iter, rel_change);
}

recon_status recon_start_features(recon_handle* h, int start, int level, float* feat) {
  if (!h || !feat || start < RECON_START_PLAIN || start > RECON_START_FFTA || level < 0 || level > 2)
    return RECON_ERR_INVALID_ARG;
  if (h->n % (1 << level) != 0) return RECON_ERR_UNSUPPORTED;
  if (h->state < ST_SMOOTHED || !h->delta_real_valid) return RECON_ERR_STATE;
  RG_CUDA(timed(h, RECON_K_OTHER, 0.0, [&] {
    return launch_features(reinterpret_cast<const float*>(h->V[2].M), h->geo, level, feat, h->st); }));
  {
    SArgs a = sargs(h);
    for (int q = 0; q < 3; ++q) a.f[q] = h->V[q];
    a.d_is_k = h->d_is_k;
    RG_TRY(run_s(h, S_DELTA, 1, AX_Y, a));
    h->d_is_k = 1;
  }
  ZArgs za = zargs(h);
  for (int q = 0; q < 3; ++q) za.f[q] = h->V[q];
  za.cform = cform(h);
  RG_TRY(xpass(h, S_INV, 3, h->V, za.cform));
  za.coef = (float)(1.0 - start_coefficient(start, h->p.f / h->p.b));
  za.u_out = reinterpret_cast<float*>(h->V[0].M);
  RG_TRY(run_z(h, Z_RADIAL, 3, za));
  RG_CUDA(timed(h, RECON_K_OTHER, 0.0, [&] {
    return launch_radial(reinterpret_cast<const float*>(h->V[0].M), nullptr, nullptr, h->geo, 1.f, level, feat, 5, 4,
                         level ? h->ucoarse : nullptr, h->st); }));
  h->delta_real_valid = 0;
  h->warm_level = level;
  return RECON_OK;
}

recon_status recon_get_radial(recon_handle* h, int level, float* u) {
  if (!h || !u || level < 0 || level > 2) return RECON_ERR_INVALID_ARG;
  if (h->n % (1 << level) != 0) return RECON_ERR_UNSUPPORTED;
  if (h->state != ST_ITERATED) return RECON_ERR_STATE;
  RG_CUDA(timed(h, RECON_K_OTHER, 0.0, [&] {
    return launch_radial(reinterpret_cast<const float*>(h->V[0].M), reinterpret_cast<const float*>(h->V[1].M),
                         reinterpret_cast<const float*>(h->V[2].M), h->geo, 1.f, level, u, 1, 0, nullptr, h->st); }));
  return RECON_OK;
}

recon_status recon_get_trace(recon_handle* h, double* rel, int cap, int* n) {
  if (!h || (cap > 0 && !rel)) return RECON_ERR_INVALID_ARG;
  const int m = (int)h->trace.size();
  for (int i = 0; i < m && i < cap; ++i) rel[i] = h->trace[i];
  if (n) *n = m;
  return RECON_OK;
}

recon_status recon_shift(recon_handle* h, const recon_catalog* cat, int is_galaxy, float* shift_out,
                         double* pos_out, int out_on_device) {
  if (!h) return RECON_ERR_INVALID_ARG;
  RG_TRY(check_catalog(cat));
  if (cat->n > 0 && !shift_out) return RECON_ERR_INVALID_ARG;
  if (h->state != ST_ITERATED) return RECON_ERR_STATE;
  ShiftArgs a{};
  for (int q = 0; q < 3; ++q) a.psi[q] = reinterpret_cast<const float*>(h->V[q].M);
  a.n = h->n;
  a.scale = (double)h->n / h->L;
  a.L = h->L;
  a.is_galaxy = is_galaxy ? 1 : 0;
  a.f = (float)h->p.f;
  a.los_mode = h->p.los_mode;
  a.los = h->geo.los;
  a.off = h->cur_off;
  a.H = (float)(h->L / h->n);
  a.periodic = h->p.periodic;
  const size_t es = elem_size(cat->dtype);
  BrickShiftArgs ba{};
  for (int q = 0; q < 3; ++q) ba.psi[q] = a.psi[q];
  ba.off = h->cur_off;
  ba.H = h->L / h->n;
  ba.is_galaxy = a.is_galaxy;
  ba.f = a.f;
  ba.los_mode = a.los_mode;
  ba.los = a.los;
  ba.periodic = a.periodic;
  ba.L = h->L;
  ba.dtype = cat->dtype == RECON_F64 ? 0 : 1;
  const bool same = h->memo.valid && cat->pos == h->memo.pos && cat->n == h->memo.n && cat->dtype == h->memo.dtype &&
                    cat->on_device == h->memo.on_device;
  if (h->reuse_sort && same && !pos_out && cat->n > 0) {
    // the deposit's brick order of this very catalogue: no second read of the positions
    float* dst = out_on_device ? shift_out : reinterpret_cast<float*>(h->bb.pre);
    ba.pos = nullptr;
    ba.pos_out = nullptr;
    ba.shift = dst;
    RG_CUDA(timed(h, RECON_K_SHIFT, (double)cat->n * (16 + 4 + 12), [&] { return brick_shift(h->bb, ba, h->st); }));
    if (!out_on_device) {
      RG_CUDA(cudaMemcpyAsync(shift_out, dst, (size_t)cat->n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->st));
      RG_CUDA(cudaStreamSynchronize(h->st));
    }
    return RECON_OK;
  }
  // with a retained brick order, other catalogues take the direct path so that it survives
  const bool sorted = h->shift_path == RECON_PATH_SORTED && !(h->reuse_sort && h->memo.valid);
  if (sorted) h->memo.valid = 0;
  const bool staged = !cat->on_device || !out_on_device;
  const long long chunk = staged ? (kStageParticles < h->bb.chunk ? kStageParticles : h->bb.chunk) : h->bb.chunk;
  if (staged && !h->copy_st) {
    RG_CUDA(cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      RG_CUDA(cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming));
      RG_CUDA(cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming));
      RG_CUDA(cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming));
    }
  }
  // Staged chunks alternate between two buffers: the copy stream brings chunk i + 1 in (and takes
  // chunk i - 1's shifts out) while the handle's stream runs chunk i's kernels.
  long long i = 0;
  for (long long p0 = 0; p0 < cat->n; p0 += chunk, ++i) {
    const long long m = (cat->n - p0 < chunk) ? cat->n - p0 : chunk;
    const int b = (int)(i & 1);
    char* sbuf = h->stage + (size_t)b * kStageParticles * kStageBytesPer;
    char* spos = sbuf;
    float* sshift = reinterpret_cast<float*>(sbuf + kStageParticles * 28);
    double* spout = reinterpret_cast<double*>(sbuf + kStageParticles * 40);
    const void* pin = (const char*)cat->pos + (size_t)p0 * 3 * es;
    if (staged && i >= 2) {
      // buffer b's previous chunk is done (kernels and copies) before it is reused
      RG_CUDA(cudaStreamWaitEvent(h->copy_st, h->ev_free[b], 0));
      RG_CUDA(cudaStreamWaitEvent(h->st, h->ev_free[b], 0));
    }
    if (!cat->on_device) {
      RG_CUDA(cudaMemcpyAsync(spos, pin, (size_t)m * 3 * es, cudaMemcpyHostToDevice, h->copy_st));
      RG_CUDA(cudaEventRecord(h->ev_in[b], h->copy_st));
      RG_CUDA(cudaStreamWaitEvent(h->st, h->ev_in[b], 0));
      pin = spos;
    }
    ba.pos = pin;
    ba.shift = out_on_device ? shift_out + 3 * p0 : sshift;
    ba.pos_out = pos_out ? (out_on_device ? pos_out + 3 * p0 : spout) : nullptr;
    if (sorted) {
      RG_CUDA(timed(h, RECON_K_SORT, (double)m * (6 * es + 28),
                    [&] { return brick_sort(h->bb, pin, cat->dtype, nullptr, m, h->st); }));
      RG_CUDA(timed(h, RECON_K_SHIFT, (double)m * (16 + 4 + 12 + (pos_out ? 3 * es + 24 : 0)),
                    [&] { return brick_shift(h->bb, ba, h->st); }));
    } else {
      a.shift = ba.shift;
      a.pos_out = ba.pos_out;
      RG_CUDA(timed(h, RECON_K_SHIFT, (double)m * (3 * es + 12 + (pos_out ? 24 : 0)),
                    [&] { return launch_shift(pin, cat->dtype, m, a, h->st); }));
    }
    if (!out_on_device) {
      RG_CUDA(cudaEventRecord(h->ev_out[b], h->st));
      RG_CUDA(cudaStreamWaitEvent(h->copy_st, h->ev_out[b], 0));
      RG_CUDA(cudaMemcpyAsync(shift_out + 3 * p0, sshift, (size_t)m * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                              h->copy_st));
      if (pos_out)
        RG_CUDA(cudaMemcpyAsync(pos_out + 3 * p0, spout, (size_t)m * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                h->copy_st));
      RG_CUDA(cudaEventRecord(h->ev_free[b], h->copy_st));
    } else if (staged) {
      RG_CUDA(cudaEventRecord(h->ev_free[b], h->st));
    }
  }
  if (staged && i > 0) {
    // the handle's stream resumes after the last copies; host memory is released on return
    for (long long k = (i >= 2 ? i - 2 : 0); k < i; ++k)
      RG_CUDA(cudaStreamWaitEvent(h->st, h->ev_free[k & 1], 0));
    RG_CUDA(cudaStreamSynchronize(h->st));
  }
  return RECON_OK;
}

recon_status recon_get_psi(recon_handle* h, float* out, int out_on_device) {
  return recon_get_field(h, RECON_FIELD_PSI, out, out_on_device);
}

recon_status recon_get_field(recon_handle* h, int which, float* out, int out_on_device) {
  if (!h || !out) return RECON_ERR_INVALID_ARG;
  const size_t nr = (size_t)h->n * h->n * h->n;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  switch (which) {
    case RECON_FIELD_RHO_G:
    case RECON_FIELD_RHO_R:
      if (h->state != ST_DEPOSITED) return RECON_ERR_STATE;
      if (which == RECON_FIELD_RHO_R && h->p.mean_density_mode == RECON_MEAN_UNIFORM) return RECON_ERR_INVALID_ARG;
      RG_CUDA(cudaMemcpyAsync(out, h->V[which == RECON_FIELD_RHO_G ? 0 : 1].M, nr * sizeof(float), kind, h->st));
      break;
    case RECON_FIELD_DELTA: {
      if (!h->delta_real_valid) return RECON_ERR_STATE;
      RG_CUDA(cudaMemcpyAsync(out, h->V[2].M, nr * sizeof(float), kind, h->st));
      if (h->p.lognormal) {
        double s = 0;
        RG_CUDA(cudaMemcpyAsync(&s, h->red + RED_SUM_LOG, sizeof(double), cudaMemcpyDeviceToHost, h->st));
        RG_CUDA(cudaStreamSynchronize(h->st));
        const float c = (float)(-s / (double)nr);
        if (out_on_device) {
          RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * nr, [&] { return launch_add_scalar(out, nr, c, h->st); }));
        } else {
          for (size_t i = 0; i < nr; ++i) out[i] += c;
        }
      }
      break;
    }
    case RECON_FIELD_DELTA_K:
      if (!h->d_is_k || h->state < ST_SMOOTHED) return RECON_ERR_STATE;
      RG_TRY(export_half(h, h->D, out));
      break;
    case RECON_FIELD_PSI:
      if (h->state != ST_ITERATED) return RECON_ERR_STATE;
      for (int q = 0; q < 3; ++q)
        RG_CUDA(cudaMemcpyAsync(out + q * nr, h->V[q].M, nr * sizeof(float), kind, h->st));
      break;
    default:
      return RECON_ERR_INVALID_ARG;
  }
  if (!out_on_device) RG_CUDA(cudaStreamSynchronize(h->st));
  return RECON_OK;
}

recon_status recon_get_scalars(recon_handle* h, double out[8]) {
  if (!h || !out) return RECON_ERR_INVALID_ARG;
  double r[RED_COUNT];
  RG_CUDA(cudaMemcpyAsync(r, h->red, sizeof(r), cudaMemcpyDeviceToHost, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));
  const double nr = (double)h->n * h->n * h->n;
  const bool uniform = h->p.mean_density_mode == RECON_MEAN_UNIFORM;
  out[0] = r[RED_SUM_WG];
  out[1] = r[RED_SUM_WR];
  out[2] = uniform ? r[RED_SUM_WG] / nr : r[RED_SUM_WG] / r[RED_SUM_WR];
  out[3] = uniform ? 0.0 : h->p.mask_frac * r[RED_SUM_WR] / r[RED_CNT_RPOS];
  out[4] = h->p.lognormal ? -r[RED_SUM_LOG] / nr : 0.0;
  out[5] = uniform ? nr : r[RED_CNT_MASK];
  out[6] = r[RED_NORM_D2];
  out[7] = r[RED_NORM_S2];
  return RECON_OK;
}

recon_status recon_fft_r2c(recon_handle* h, const float* in_real, float* out_half) {
  if (!h || !in_real || !out_half) return RECON_ERR_INVALID_ARG;
  const size_t nr = (size_t)h->n * h->n * h->n;
  h->state = ST_CREATED;
  h->warm_level = -1;
  h->d_is_k = 0;
  h->delta_real_valid = 0;
  RG_CUDA(cudaMemcpyAsync(h->V[0].M, in_real, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  ZArgs a = zargs(h);
  a.f[0] = h->V[0];
  RG_TRY(run_z(h, Z_FWD, 1, a));
  RG_TRY(xpass(h, S_FWD, 1, h->V));
  SArgs s = sargs(h);
  s.f[0] = h->V[0];
  RG_TRY(run_s(h, S_FWD, 1, AX_Y, s));
  RG_TRY(export_half(h, h->V[0], out_half));
  return RECON_OK;
}

recon_status recon_fft_c2r(recon_handle* h, const float* in_half, float* out_real) {
  if (!h || !in_half || !out_real) return RECON_ERR_INVALID_ARG;
  const size_t nr = (size_t)h->n * h->n * h->n;
  h->state = ST_CREATED;
  h->warm_level = -1;
  h->d_is_k = 0;
  h->delta_real_valid = 0;
  RG_TRY(import_half(h, in_half, h->V[0]));
  SArgs s = sargs(h);
  s.f[0] = h->V[0];
  RG_TRY(run_s(h, S_INV, 1, AX_Y, s));
  RG_TRY(xpass(h, S_INV, 1, h->V));
  ZArgs a = zargs(h);
  a.f[0] = h->V[0];
  RG_TRY(run_z(h, Z_INV, 1, a));
  RG_CUDA(cudaMemcpyAsync(out_real, h->V[0].M, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  return RECON_OK;
}

// ---- the finite-difference method of Sec. 2.1 (the paper's comparison method) ----------------
namespace {

// x . y in float64 over n values (one synchronisation).
recon_status fd_dot(recon_handle* h, const float* x, const float* y, size_t n, double* out) {
  const int blocks = kDepositBlocks;
  RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * n, [&] { return launch_dot(x, y, n, h->partials, blocks, h->st); }));
  RG_TRY(finalize(h, blocks, 1, RED_DIAG, 0));
  RG_CUDA(cudaMemcpyAsync(out, h->red + RED_DIAG, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));
  return RECON_OK;
}

// out = M^-1 in: the inverse of the periodic 7-point Laplacian through the library's FFT passes on
// the handle's first field.
recon_status fd_precond(recon_handle* h, const float* in, float* out) {
  const size_t nr = (size_t)h->n * h->n * h->n;
  RG_CUDA(cudaMemcpyAsync(h->V[0].M, in, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  ZArgs a = zargs(h);
  a.f[0] = h->V[0];
  RG_TRY(run_z(h, Z_FWD, 1, a));
  RG_TRY(xpass(h, S_FWD, 1, h->V));
  SArgs s = sargs(h);
  s.f[0] = h->V[0];
  RG_TRY(run_s(h, S_FWD, 1, AX_Y, s));
  RG_CUDA(timed(h, RECON_K_OTHER, 2.0 * cfield(h), [&] { return launch_fd_precond_k(h->V[0], h->n, h->L, h->st); }));
  RG_TRY(run_s(h, S_INV, 1, AX_Y, s));
  RG_TRY(xpass(h, S_INV, 1, h->V));
  RG_TRY(run_z(h, Z_INV, 1, a));
  RG_CUDA(cudaMemcpyAsync(out, h->V[0].M, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  return RECON_OK;
}

struct DeviceBuffer {
  void* p = nullptr;
  ~DeviceBuffer() {
    if (p) cudaFree(p);
  }
};

}  // namespace

recon_status recon_fd_solve(recon_handle* h, double tol, int max_iter, int* n_iter, double* rel_resid, float* psi_out) {
  if (!h || !psi_out || !(tol > 0) || max_iter < 1) return RECON_ERR_INVALID_ARG;
  if (h->state < ST_SMOOTHED || !h->delta_real_valid) return RECON_ERR_STATE;
  const size_t nr = (size_t)h->n * h->n * h->n;
  DeviceBuffer buf;
  if (cudaMalloc(&buf.p, 9 * nr * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return RECON_ERR_OOM;
  }
  float* v0 = static_cast<float*>(buf.p);
  float *x = v0, *r = v0 + nr, *rh = v0 + 2 * nr, *p = v0 + 3 * nr, *v = v0 + 4 * nr, *ph = v0 + 5 * nr,
        *sv = v0 + 6 * nr, *sh = v0 + 7 * nr, *t = v0 + 8 * nr;
  FDArgs fa{};
  fa.n = h->n;
  fa.g = h->L / h->n;
  fa.beta = h->p.f / h->p.b;
  fa.los_mode = h->p.los_mode;
  fa.los = make_double3(h->geo.los.x, h->geo.los.y, h->geo.los.z);
  fa.off = h->cur_off;
  // right-hand side delta / b (the lognormal constant added back, as recon_get_field does)
  RG_CUDA(cudaMemcpyAsync(rh, h->V[2].M, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  if (h->p.lognormal) {
    double sl = 0;
    RG_CUDA(cudaMemcpyAsync(&sl, h->red + RED_SUM_LOG, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    RG_CUDA(cudaStreamSynchronize(h->st));
    RG_CUDA(launch_add_scalar(rh, nr, (float)(-sl / (double)nr), h->st));
  }
  RG_CUDA(cudaMemsetAsync(x, 0, nr * sizeof(float), h->st));
  RG_CUDA(launch_fd_sub(r, x, rh, -1.0 / h->p.b, nr, h->st));     // r = 0 + delta / b
  RG_CUDA(cudaMemcpyAsync(rh, r, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  double bnorm2 = 0;
  RG_TRY(fd_dot(h, r, r, nr, &bnorm2));
  const double bnorm = std::sqrt(bnorm2);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0, res = bnorm > 0 ? 1.0 : 0.0;
  int it = 0;
  // BiCGStab, right-preconditioned (A M^-1 y = b, x = M^-1 y)
  while (res > tol && it < max_iter) {
    ++it;
    double rho = 0;
    RG_TRY(fd_dot(h, rh, r, nr, &rho));
    if (it == 1) {
      RG_CUDA(cudaMemcpyAsync(p, r, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    } else {
      RG_CUDA(launch_fd_dir(p, r, v, (rho / rho_old) * (alpha / omega), omega, nr, h->st));
    }
    RG_TRY(fd_precond(h, p, ph));
    RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * nr, [&] { return launch_fd_apply(ph, v, fa, h->st); }));
    double rv = 0;
    RG_TRY(fd_dot(h, rh, v, nr, &rv));
    alpha = rho / rv;
    RG_CUDA(launch_fd_sub(sv, r, v, alpha, nr, h->st));
    double s2 = 0;
    RG_TRY(fd_dot(h, sv, sv, nr, &s2));
    if (std::sqrt(s2) / bnorm <= tol) {
      RG_CUDA(launch_fd_acc(x, ph, ph, alpha, 0.0, nr, h->st));
      res = std::sqrt(s2) / bnorm;
      break;
    }
    RG_TRY(fd_precond(h, sv, sh));
    RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * nr, [&] { return launch_fd_apply(sh, t, fa, h->st); }));
    double ts = 0, tt = 0;
    RG_TRY(fd_dot(h, t, sv, nr, &ts));
    RG_TRY(fd_dot(h, t, t, nr, &tt));
    omega = tt > 0 ? ts / tt : 0.0;
    RG_CUDA(launch_fd_acc(x, ph, sh, alpha, omega, nr, h->st));
    RG_CUDA(launch_fd_sub(r, sv, t, omega, nr, h->st));
    double r2 = 0;
    RG_TRY(fd_dot(h, r, r, nr, &r2));
    res = std::sqrt(r2) / bnorm;
    if (!std::isfinite(res)) return RECON_ERR_NONFINITE;
    rho_old = rho;
    if (omega == 0.0) break;
  }
  // the true residual |A x - b| / |b| and Psi = -grad phi
  RG_CUDA(launch_fd_apply(x, t, fa, h->st));
  RG_CUDA(launch_fd_sub(t, t, rh, 1.0, nr, h->st));
  double tr2 = 0;
  RG_TRY(fd_dot(h, t, t, nr, &tr2));
  RG_CUDA(timed(h, RECON_K_OTHER, 16.0 * nr, [&] { return launch_fd_gradient(x, psi_out, fa, h->st); }));
  RG_CUDA(cudaStreamSynchronize(h->st));
  if (n_iter) *n_iter = it;
  const double true_res = bnorm > 0 ? std::sqrt(tr2) / bnorm : 0.0;
  if (rel_resid) *rel_resid = true_res;
  h->delta_real_valid = 1;   // the real delta (third field) is untouched; only the first field was used
  return res > tol ? RECON_ERR_NOT_CONVERGED : RECON_OK;
}

// ---- the paper's front end (Sec. 3.2): radial number density and FKP weights ------------------
recon_status recon_radial_nbar(recon_handle* h, const recon_catalog* cat, int nbins, double rmin, double rmax,
                               double sky_area, double* nbar) {
  if (!h || !nbar || nbins < 1 || nbins > 4096 || !(rmax > rmin) || !(rmin >= 0) || !(sky_area > 0))
    return RECON_ERR_INVALID_ARG;
  RG_TRY(check_catalog(cat));
  if (cat->n > 0 && !cat->on_device) return RECON_ERR_INVALID_ARG;
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(h->partials);
  RG_CUDA(cudaMemsetAsync(counts, 0, (size_t)nbins * sizeof(unsigned long long), h->st));
  const double3 obs = make_double3(h->p.observer[0], h->p.observer[1], h->p.observer[2]);
  RG_CUDA(timed(h, RECON_K_OTHER, (double)cat->n * 3 * elem_size(cat->dtype), [&] {
    return launch_radial_hist(cat->pos, cat->dtype, cat->n, obs, rmin, rmax, nbins, counts, h->st); }));
  std::vector<unsigned long long> c(nbins);
  RG_CUDA(cudaMemcpyAsync(c.data(), counts, nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));
  const double dr = (rmax - rmin) / nbins;
  for (int b = 0; b < nbins; ++b) {
    const double lo = rmin + b * dr, hi = rmin + (b + 1) * dr;
    nbar[b] = (double)c[b] / (sky_area * (hi * hi * hi - lo * lo * lo) / 3.0);
  }
  return RECON_OK;
}

recon_status recon_fkp_weights(recon_handle* h, const recon_catalog* cat, int nbins, double rmin, double rmax,
                               const double* nbar, double P0, float* w_out) {
  if (!h || !nbar || nbins < 1 || nbins > 4096 || !(rmax > rmin) || !(P0 >= 0)) return RECON_ERR_INVALID_ARG;
  RG_TRY(check_catalog(cat));
  if (cat->n > 0 && (!cat->on_device || !w_out)) return RECON_ERR_INVALID_ARG;
  double* dnb = h->partials;
  RG_CUDA(cudaMemcpyAsync(dnb, nbar, nbins * sizeof(double), cudaMemcpyHostToDevice, h->st));
  const double3 obs = make_double3(h->p.observer[0], h->p.observer[1], h->p.observer[2]);
  RG_CUDA(timed(h, RECON_K_OTHER, (double)cat->n * (3 * elem_size(cat->dtype) + 4), [&] {
    return launch_fkp(cat->pos, cat->dtype, cat->n, obs, rmin, rmax, nbins, dnb, P0, w_out, h->st); }));
  RG_CUDA(cudaStreamSynchronize(h->st));   // nbar is read from the caller's host memory
  return RECON_OK;
}

// ---- the paper's diagnostics (Sec. 4.1, Eq. Helmholtz; Sec. 4.3 and 5.2, Eq. ratio) ----------
namespace {

recon_status ratio_result(recon_handle* h, int blocks, double out[4]) {
  RG_TRY(finalize(h, blocks, 4, RED_DIAG, 0));
  double r[4];
  RG_CUDA(cudaMemcpyAsync(r, h->red + RED_DIAG, sizeof(r), cudaMemcpyDeviceToHost, h->st));
  RG_CUDA(cudaStreamSynchronize(h->st));
  const double k = r[0];
  const double mean = k > 0 ? r[1] / k : 0.0;
  const double var = k > 0 ? r[2] / k - mean * mean : 0.0;
  out[0] = mean;
  out[1] = var > 0 ? std::sqrt(var) : 0.0;
  out[2] = r[3] > 0 ? 1.0 - k / r[3] : 0.0;
  out[3] = k;
  return RECON_OK;
}

}  // namespace

recon_status recon_ratio_stats(recon_handle* h, const float* num, const float* den, int64_t n, double lo, double hi,
                               double out[4]) {
  if (!h || !out || n < 0 || (n > 0 && (!num || !den)) || !(lo <= hi)) return RECON_ERR_INVALID_ARG;
  const int blocks = kDepositBlocks;
  RG_CUDA(timed(h, RECON_K_OTHER, 8.0 * n, [&] {
    return launch_ratio(num, den, (size_t)n, lo, hi, h->partials, blocks, h->st); }));
  return ratio_result(h, blocks, out);
}

recon_status recon_radial_ratio(recon_handle* h, const float* psi_num, const float* psi_den, const recon_catalog* cat,
                                double lo, double hi, double out[4]) {
  if (!h || !psi_num || !psi_den || !out || !(lo <= hi)) return RECON_ERR_INVALID_ARG;
  RG_TRY(check_catalog(cat));
  if (cat->n > 0 && !cat->on_device) return RECON_ERR_INVALID_ARG;
  const size_t nr = (size_t)h->n * h->n * h->n;
  RatioArgs a{};
  for (int q = 0; q < 3; ++q) {
    a.num[q] = psi_num + q * nr;
    a.den[q] = psi_den + q * nr;
  }
  a.n = h->n;
  a.scale = (double)h->n / h->L;
  a.los_mode = h->p.los_mode;
  a.los = h->geo.los;
  a.off = h->cur_off;
  a.H = (float)(h->L / h->n);
  a.lo = lo;
  a.hi = hi;
  a.partials = h->partials;
  const int blocks = kDepositBlocks;
  RG_CUDA(timed(h, RECON_K_OTHER, (double)cat->n * 3 * elem_size(cat->dtype), [&] {
    return cat->n > 0 ? launch_radial_ratio(cat->pos, cat->dtype, cat->n, a, blocks, h->st)
                      : cudaMemsetAsync(h->partials, 0, (size_t)blocks * 4 * sizeof(double), h->st); }));
  return ratio_result(h, blocks, out);
}

recon_status recon_helmholtz_x(recon_handle* h, const float* psi_x, float* grad_a, float* curl_b) {
  if (!h || !psi_x || !grad_a || !curl_b) return RECON_ERR_INVALID_ARG;
  const size_t nr = (size_t)h->n * h->n * h->n;
  h->state = ST_CREATED;
  h->warm_level = -1;
  h->d_is_k = 0;
  h->delta_real_valid = 0;
  // Psi_x(k) in the first field (forward z, x, y passes)
  RG_CUDA(cudaMemcpyAsync(h->V[0].M, psi_x, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  {
    ZArgs a = zargs(h);
    a.f[0] = h->V[0];
    RG_TRY(run_z(h, Z_FWD, 1, a));
    RG_TRY(xpass(h, S_FWD, 1, h->V));
    SArgs s = sargs(h);
    s.f[0] = h->V[0];
    RG_TRY(run_s(h, S_FWD, 1, AX_Y, s));
  }
  for (int j = 0; j < 3; ++j) {
    RG_CUDA(timed(h, RECON_K_OTHER, 2.0 * cfield(h), [&] { return launch_helmholtz_k(h->V[0], h->V[1], j, h->geo, h->st); }));
    SArgs s = sargs(h);
    s.f[0] = h->V[1];
    RG_TRY(run_s(h, S_INV, 1, AX_Y, s));
    RG_TRY(xpass(h, S_INV, 1, h->V + 1));
    ZArgs a = zargs(h);
    a.f[0] = h->V[1];
    RG_TRY(run_z(h, Z_INV, 1, a));
    RG_CUDA(cudaMemcpyAsync(grad_a + j * nr, h->V[1].M, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    RG_CUDA(timed(h, RECON_K_OTHER, 12.0 * nr, [&] {
      return launch_solenoidal(psi_x, grad_a + j * nr, curl_b + j * nr, nr, j, h->st); }));
  }
  return RECON_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Batches as CUDA graphs (recon_batch_run): each mock appends its whole reconstruction to a graph
// (its own, or the one graph of the whole batch), with the handle of its size class.  A class's
// mocks run one after another on the class's buffers; the host waits once, for the whole batch.
// ------------------------------------------------------------------------------------------------
namespace rg {

#define RG_GTRY(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return RECON_ERR_CUDA;                                       \
    }                                                              \
  } while (0)

recon_status batch_append(recon_handle* h, cudaGraph_t top, cudaGraphNode_t* last, const BatchJob& job) {
  recon_batch_item& it = *job.item;
  if (it.tol < 0 || it.max_iter < 1 || it.max_iter > kMaxTrace || it.start < RECON_START_PLAIN ||
      it.start > RECON_START_FFTA)
    return RECON_ERR_INVALID_ARG;
  if (!it.gal.on_device || (it.ran.n > 0 && !it.ran.on_device) ||
      ((it.shift_gal || it.shift_ran) && !it.out_on_device))
    return RECON_ERR_UNSUPPORTED;   // host memory cannot be read or written inside the graph
  if (!h->cap_stream) RG_GTRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const cudaStream_t user = h->st;
  h->st = h->cap_stream;
  const bool uniform = it.params.mean_density_mode == RECON_MEAN_UNIFORM;
  cudaGraph_t pre = nullptr, post = nullptr;
  recon_status rs = RECON_OK;
  do {
    // deposit, smoothing, loop state and the start
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) { rs = RECON_ERR_CUDA; break; }
    rs = [&]() -> recon_status {
      RG_GTRY(launch_stamp(&job.slot->t0, h->st));
      apply_config(h, &it.params, job.taps_dev, job.t0, job.ntap, job.off_dev);
      RG_TRY(recon_deposit(h, &it.gal, uniform ? nullptr : &it.ran));
      RG_TRY(recon_smooth(h));
      h->trace.clear();
      h->delta_real_valid = 0;
      RG_GTRY(launch_loop_init(h->loop, it.tol, it.max_iter, h->st));
      StartSpec sp;
      sp.coef0 = (float)(1.0 - start_coefficient(it.start, it.params.f / it.params.b));
      return run_start(h, sp);
    }();
    cudaError_t e = cudaStreamEndCapture(h->st, &pre);
    if (rs != RECON_OK) break;
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraphNode_t npre = nullptr, ncond = nullptr, npost = nullptr;
    if ((e = cudaGraphAddChildGraphNode(&npre, top, *last ? last : nullptr, *last ? 1 : 0, pre)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    // the updates of Eq. iterative as a conditional WHILE node (device-side stopping test)
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, top, 1, cudaGraphCondAssignDefault)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if ((e = cudaGraphAddNode(&ncond, top, &npre, nullptr, 1, &np)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    if ((e = cudaStreamBeginCaptureToGraph(h->st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    rs = iterate_body(h, cond);
    cudaGraph_t body_out = nullptr;
    e = cudaStreamEndCapture(h->st, &body_out);
    if (rs != RECON_OK) break;
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    h->d_is_k = 1;
    h->state = ST_ITERATED;
    // the loop's outcome, the shifts, the end stamp
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) { rs = RECON_ERR_CUDA; break; }
    rs = [&]() -> recon_status {
      RG_GTRY(launch_loop_record(h->loop, job.slot, h->st));
      if (it.shift_gal && it.gal.n > 0) RG_TRY(recon_shift(h, &it.gal, 1, it.shift_gal, nullptr, 1));
      if (!uniform && it.shift_ran && it.ran.n > 0) RG_TRY(recon_shift(h, &it.ran, 0, it.shift_ran, nullptr, 1));
      RG_GTRY(launch_stamp(&job.slot->t1, h->st));
      return RECON_OK;
    }();
    e = cudaStreamEndCapture(h->st, &post);
    if (rs != RECON_OK) break;
    if (e != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    if ((e = cudaGraphAddChildGraphNode(&npost, top, &ncond, 1, post)) != cudaSuccess) { h->err = cudaGetErrorString(e); rs = RECON_ERR_CUDA; break; }
    *last = npost;
  } while (0);
  if (pre) cudaGraphDestroy(pre);     // child nodes hold their own copies
  if (post) cudaGraphDestroy(post);
  h->st = user;
  return rs;
}

void batch_restore(recon_handle* h) {
  h->cur_taps = h->taps;
  h->cur_off = h->off;
  h->geo.off = h->off;
  ++h->epoch;
  h->state = ST_CREATED;
}

}  // namespace rg
