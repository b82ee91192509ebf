// inst_f.cu: kernel instantiations for mesh sides 256 and 384 in the alternative radix order
// (smallest radix first: 4 8 8 and 6 8 8, their z plans 4 4 8 and 3 8 8).
#define RG_RADIX_ORDER 1
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_256_order1() { return MeshImpl<256>::table(); }
const MeshKernels* mesh_kernels_384_order1() { return MeshImpl<384>::table(); }
}  // namespace rg
