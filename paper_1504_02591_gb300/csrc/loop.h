// loop.h: device-side convergence test for the graph-captured iteration.
#pragma once
#include <cuda_runtime.h>

#include "types.h"

namespace rg {

cudaError_t launch_loop_init(LoopState* s, double tol, int max_iter, cudaStream_t st);
cudaError_t launch_loop_decide(LoopState* s, const double* red, cudaGraphConditionalHandle cond, cudaStream_t st);

}  // namespace rg
