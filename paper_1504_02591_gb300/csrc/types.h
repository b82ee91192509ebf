// types.h: argument blocks shared by the host orchestration and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rg {

// A field on the mesh.  In configuration space M holds N^3 float32 [ix][iy][iz].  On the r2c half
// grid M holds the kz = 0..N/2-1 planes as N*N*(N/2) float2 [kx][ky][kz] (same bytes as the real
// field, so every row stays 16-byte aligned) and Q holds the kz = N/2 (Nyquist) plane, N*N float2
// [kx][ky].
struct Field {
  float2* M;
  float2* Q;
};

// Slots of the float64 reduction block kept on the device.
enum RedSlot {
  RED_SUM_WG = 0,      // sum of galaxy weights
  RED_SUM_WR = 1,      // sum of random weights
  RED_SUM_RPOS = 2,    // (unused) partner slot of RED_CNT_RPOS in the reduction
  RED_CNT_RPOS = 3,    // number of nodes that received random mass in the deposit
  RED_SUM_LOG = 4,     // sum over nodes of ln(max(1 + delta, floor)) (lognormal mode)
  RED_CNT_MASK = 5,    // number of nodes inside the survey mask
  RED_NORM_D2 = 6,     // Parseval sum for |dPsi|^2 of the last iteration
  RED_NORM_S2 = 7,     // Parseval sum for |Psi|^2 of the last iteration
  RED_DIAG = 8,        // 4 slots: ratio statistics (kept count, sum, sum of squares, points)
  RED_COUNT = 12
};

struct Geometry {
  int n;                  // mesh side
  float kf;               // 2 pi / L
  float inv_n3;           // 1 / N^3
  int los_mode;           // 0 radial, 1 fixed
  float3 los;             // fixed LOS unit vector
  const float* off;       // 3 N node offsets from the observer: x_i - o_a, per axis a (radial)
};

enum ZMode { Z_FWD = 0, Z_INV = 1, Z_DELTA = 2, Z_PROJ = 3, Z_FINAL = 4, Z_USTART = 5, Z_RADIAL = 6, Z_WARM = 7 };
enum SMode { S_FWD = 0, S_INV = 1, S_DELTA = 3, S_ITER = 4 };
enum Axis { AX_X = 0, AX_Y = 1 };

struct ZArgs {
  Field f[3];             // fields transformed in place
  Geometry g;
  const float2* tw;       // exp(-2 pi i m / N), m < N
  const float2* tab;      // stage twiddles of the N/2-point plan
  double* partials;       // per-block reduction partials (4 per block)
  const double* red;      // reduction block (read by Z_DELTA)
  float coef;             // Z_PROJ: (1 - c) multiplier of the projection
  // Z_DELTA
  Field dout;             // delta on the (z-transformed) half grid
  float* delta_real;      // optional real copy of delta
  double mask_frac;
  int uniform;            // delta from rho_bar = sum w_g / N^3
  int lognormal;
  const float* taps;      // z factor of the Gaussian smoothing: g[t0 .. t0 + ntap - 1]
  int ntap;
  int t0;
  const int* loop_flag;   // Z_PROJ in a device-driven loop: 1 = converged, write the real Psi
  const float* u_in;      // Z_USTART / Z_WARM: radial displacement u (real N^3); P = u r is transformed
  float* u_out;           // Z_RADIAL: coef (Psi.r), real N^3 (may alias f[0])
  // Z_WARM: u += trilinear upsampling of (corr - ucoarse), both on the (N >> clevel)^3 grid
  const float* corr;
  const float* ucoarse;
  int clevel;
  int generic;            // Z_PROJ: the generic staged kernel instead of the register-fused one
  int ybeg, ycount;       // register-fused passes: only the rows of y-planes [ybeg, ybeg + ycount)
                          // (ycount 0: every row)
  // Z_PROJ of the register-fused path while the loop runs: the inverse x pass handed over
  // C = dx Psi_x + dy Psi_y in f[0] and Psi_z in wf (two fields read, not three)
  int cform;
  Field wf;
};

// Tensor maps of the register-fused source update's four inputs (A, P_y, delta(k), S) over the
// half grid M [kx][ky][kz < N/2] (N = 512), built on the host; passed to the kernel by value.
struct KIterMaps {
  CUtensorMap m[4];
};

struct SArgs {
  Field f[3];             // fields transformed in place
  Geometry g;
  const float2* tab;      // stage twiddles of the N-point plan
  double* partials;       // per-block partials (2 per block, S_ITER)
  const double* red;      // reduction block (S_DELTA reads the lognormal sum)
  Field dk;               // delta: partially transformed (S_DELTA input) / k-space (S_ITER)
  Field sbuf;             // stored source S of the previous iteration
  float inv_b;            // 1 / b
  float beta;             // f / b
  int d_is_k;             // S_DELTA: dk is already fully transformed
  int lognormal;          // S_DELTA: subtract the lognormal constant at k = 0
  const int* skip_flag;   // plain passes: do nothing when *skip_flag != 0 (device-driven loop)
  int narrow;             // plain x passes: 8-column instead of 16-column tiles
  int generic;            // k-space update: the generic staged kernel instead of the register-fused one
  int ybeg, ycount;       // paired x passes: only the lines of y-planes [ybeg, ybeg + ycount)
                          // (ycount 0: every line; both multiples of the tile width)
  const KIterMaps* tmaps; // host memory: the source update streams its inputs by TMA (N = 512)
  // paired inverse x pass (N = 512) unless loop_flag && *loop_flag == 1 (the device loop has just
  // converged): leave C = dx Psi_x + dy Psi_y in f[0] and Psi_z in wf for the projection pass,
  // instead of Psi_x, Psi_y, Psi_z in f[0..2]
  int cform;
  Field wf;
  const int* loop_flag;
};

// State of the device-driven iteration (in the workspace).
constexpr int kMaxTrace = 1024;
struct LoopState {
  int flag;               // 0 running, 1 converged (final pass pending), 2 non-finite norms
  int it;                 // updates done
  int max_iter;
  int pad;
  double tol;
  double trace[kMaxTrace];
};

// Result of one mock of a batch graph, written on the device: the loop's outcome and globaltimer
// stamps (ns) at the start and end of the mock's work.
struct BatchSlot {
  int flag;               // LoopState::flag at the end of the mock's iteration
  int it;                 // updates done
  double rel;             // last |dPsi| / |Psi|
  unsigned long long t0, t1;
};

// Kernels of one mesh size (one table per supported N).
struct MeshKernels {
  int n;
  int z_blocks;           // upper bound of a Z pass grid (rows / warps per CTA)
  int s_blocks;           // CTAs of a strided pass
  int tab_s, tab_z;       // stage-twiddle table lengths (N-point and N/2-point plans)
  int kspace_fused;       // register-fused k-space passes with paired vector x passes (unless the
                          // generic option is set): 7 field transfers per y pass, 5 per x pass
  // persistent Z pass; *grid_out receives the number of CTAs launched (its reduction partials)
  cudaError_t (*zpass)(int mode, int nc, const ZArgs& a, cudaStream_t st, int* grid_out);
  cudaError_t (*spass)(int mode, int nc, int axis, const SArgs& a, cudaStream_t st);
  cudaError_t (*build_tables)(const float2* tw, float2* tabS, float2* tabZ, cudaStream_t st);
};

const MeshKernels* mesh_kernels(int n);

}  // namespace rg
