// inst_d.cu: kernel instantiations for mesh sides 512.
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_512() { return MeshImpl<512>::table(); }
}  // namespace rg
