// loop.cu: the convergence test of the iteration (Sec. 5.1) as device kernels, so that the whole
// loop can run inside one CUDA graph (a conditional WHILE node) without returning to the host.
#include "loop.h"

namespace rg {

__global__ void loop_init_kernel(LoopState* s, double tol, int max_iter) {
  s->flag = 0;
  s->it = 0;
  s->max_iter = max_iter;
  s->tol = tol;
}

// After the norms of one update: record rel = |dPsi|/|Psi|, and stop the loop (condition 0) once
// rel < tol after at least two updates, at max_iter, or on non-finite norms.
__global__ void loop_decide_kernel(LoopState* s, const double* red, cudaGraphConditionalHandle cond) {
  const double d2 = red[RED_NORM_D2], s2 = red[RED_NORM_S2];
  const int it = s->it;
  if (!isfinite(d2) || !isfinite(s2)) {
    s->flag = 2;
    cudaGraphSetConditional(cond, 0);
    return;
  }
  const double rel = s2 > 0.0 ? sqrt(d2 / s2) : 0.0;
  if (it < kMaxTrace) s->trace[it] = rel;
  s->it = it + 1;
  if ((it + 1 >= 2 && rel < s->tol) || it + 1 >= s->max_iter) {
    s->flag = 1;
    cudaGraphSetConditional(cond, 0);
  }
}

cudaError_t launch_loop_init(LoopState* s, double tol, int max_iter, cudaStream_t st) {
  loop_init_kernel<<<1, 1, 0, st>>>(s, tol, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_loop_decide(LoopState* s, const double* red, cudaGraphConditionalHandle cond, cudaStream_t st) {
  loop_decide_kernel<<<1, 1, 0, st>>>(s, red, cond);
  return cudaGetLastError();
}

__global__ void stamp_kernel(unsigned long long* t) {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  *t = v;
}

__global__ void loop_record_kernel(const LoopState* s, BatchSlot* out) {
  const int it = s->it;
  out->flag = s->flag;
  out->it = it;
  out->rel = (it > 0 && it <= kMaxTrace) ? s->trace[it - 1] : 0.0;
}

cudaError_t launch_stamp(unsigned long long* t, cudaStream_t st) {
  stamp_kernel<<<1, 1, 0, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_loop_record(const LoopState* s, BatchSlot* out, cudaStream_t st) {
  loop_record_kernel<<<1, 1, 0, st>>>(s, out);
  return cudaGetLastError();
}

}  // namespace rg
