// inst_e.cu: kernel instantiations for mesh sides 1024.
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_1024() { return MeshImpl<1024>::table(); }
}  // namespace rg
