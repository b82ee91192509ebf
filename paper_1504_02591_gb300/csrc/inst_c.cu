// inst_c.cu: kernel instantiations for mesh sides 384.
#include "passes.cuh"
namespace rg {
const MeshKernels* mesh_kernels_384() { return MeshImpl<384>::table(); }
}  // namespace rg
