// unet_tc.h: the tensor-core (tcgen05) forward convolution of the warm-start U-Net.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace rg {
namespace tc {

// How one periodic 3x3x3 convolution layer maps onto tcgen05.mma (kind::f16, bf16 in, f32 accumulate).
//
// Voxel tiles are runs of `zlen` voxels along z.  A CTA owns bx x by tiles; their input halo (the
// tiles' voxels plus one voxel on each side, and two extra along z) is staged in shared memory as
// one plane per group of 8 input channels, 16 bytes per voxel.  A run of 8 consecutive voxels of one
// channel group is then exactly one 8x16-byte core matrix, so the operand of every tap is a
// descriptor pointing into the halo at the tap's offset: no im2col copy is made.
//
// orient 0 (z runs of 128):  D[voxel, cout] += A[voxel, k] B[cout, k], M = 128, N = cout rounded to 16.
// orient 1 (z runs of 64):   D[cout, voxel] += W[cout, k] X[voxel, k], M = 128 (rows >= cout unused),
//                            N = 64.
// mode 0: K = 16 is two channel groups of one tap (27 MMAs per pair of groups);
// mode 1: K = 16 is one channel group at two neighbouring z taps (dz = -1,0 and +1,+2 with the
//         +2 weights zero; 18 MMAs per group), used when the number of groups is odd.
struct ConvPlan {
  int orient = 0, mode = 0;
  int n = 0;              // grid side of the output
  int c0 = 0, up0 = 0;    // first input: channels (multiple of 8), stored on the n/2 grid when up0
  int c1 = 0;             // second input (concatenated after the first), channels (multiple of 8) or 0
  int cin = 0, cout = 0;  // the layer's weight shape w[27][cin][cout] (cin <= c0 + c1)
  int gpc = 0, nchunk = 0, nmma = 0;
  int rows = 0, N = 0;    // weight-tile rows, MMA N
  int zlen = 0, hz = 0, bx = 0, by = 0;
  int tmem_cols = 0;
  size_t halo_bytes = 0, wts_bytes = 0, smem = 0;
  size_t packed_elems = 0;
  int grid = 0, nblocks = 0;
};

// Fills *p for a layer on an n^3 grid; false when the layer is not on the tensor-core path
// (n neither 64 nor a multiple of 128, channel counts not multiples of 8, or tiles that do not fit).
bool plan_conv(int n, int c0, int up0, int c1, int cin, int cout, ConvPlan* p);

// Reorders w[27][cin][cout] (bf16) into the per-chunk shared-memory image of the weight tiles.
cudaError_t pack_weights(const ConvPlan& p, const __nv_bfloat16* w, __nv_bfloat16* out, cudaStream_t st);

struct ConvIO {
  const __nv_bfloat16* src0 = nullptr;
  const __nv_bfloat16* src1 = nullptr;
  const __nv_bfloat16* wpack = nullptr;
  const float* bias = nullptr;
  __nv_bfloat16* out = nullptr;        // [v][cout] bf16, ReLU applied (unused with a head)
  // optional fused 1x1 head (orient 0): yout[v] = head_b + sum_c bf16(relu(.))_c head_w[c] + res[v*res_stride]
  const __nv_bfloat16* head_w = nullptr;
  const float* head_b = nullptr;
  const float* res = nullptr;
  int res_stride = 0;
  float* yout = nullptr;
  int* err = nullptr;                  // set non-zero when a wait on the tensor-core pipeline times out
};

cudaError_t conv_forward(const ConvPlan& p, const ConvIO& io, cudaStream_t st);

}  // namespace tc
}  // namespace rg
