// batch_graph.h: internal interface between the batch scheduler (batch.cu) and the handle
// (recon.cu) for running many mocks as CUDA graphs.
#pragma once
#include <vector>

#include "../../include/recon.h"
#include "types.h"

namespace rg {

// Smoothing and line-of-sight tables of one parameter set (see recon.cu).
void config_tables(int n, const recon_params* p, std::vector<float>& taps, int* t0, int* ntap,
                   std::vector<float>& off);

// One mock of a batch graph: its item (device catalogues and outputs), its tables already in
// device memory, and its result slot.
struct BatchJob {
  recon_batch_item* item;
  const float* taps_dev;
  int t0, ntap;
  const float* off_dev;
  BatchSlot* slot;
};

// Append the whole reconstruction of job (deposit -> smooth -> start -> iteration as a
// conditional WHILE node -> shifts) to the graph `top` after node *last (none if null), using the
// handle's buffers; *last becomes the job's final node.  Nothing runs until the graph is launched.
recon_status batch_append(recon_handle* h, cudaGraph_t top, cudaGraphNode_t* last, const BatchJob& job);

// Point the handle back at its own tables after a batch graph was built with it.
void batch_restore(recon_handle* h);

}  // namespace rg
