// loop.h: device-side convergence test for the graph-captured iteration.
#pragma once
#include <cuda_runtime.h>

#include "types.h"

namespace rg {

cudaError_t launch_loop_init(LoopState* s, double tol, int max_iter, cudaStream_t st);
cudaError_t launch_loop_decide(LoopState* s, const double* red, cudaGraphConditionalHandle cond, cudaStream_t st);
// Batch graphs: the device's globaltimer (ns) into *t, and the loop's outcome into a slot.
cudaError_t launch_stamp(unsigned long long* t, cudaStream_t st);
cudaError_t launch_loop_record(const LoopState* s, BatchSlot* out, cudaStream_t st);

}  // namespace rg
