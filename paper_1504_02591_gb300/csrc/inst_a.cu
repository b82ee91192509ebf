// inst_a.cu: kernel instantiations for mesh sides 32 48 64 96.
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_32() { return MeshImpl<32>::table(); }
const MeshKernels* mesh_kernels_48() { return MeshImpl<48>::table(); }
const MeshKernels* mesh_kernels_64() { return MeshImpl<64>::table(); }
const MeshKernels* mesh_kernels_96() { return MeshImpl<96>::table(); }
}  // namespace rg
