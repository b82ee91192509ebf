// inst_b.cu: kernel instantiations for mesh sides 128 256.
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_128() { return MeshImpl<128>::table(); }
const MeshKernels* mesh_kernels_256() { return MeshImpl<256>::table(); }
}  // namespace rg
