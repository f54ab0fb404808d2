// CUDA-event timing of the two passes over X of every nnTD sweep (the
// dominant kernels), for nnc_profile_enable / nnc_profile_read.
//
// The sweep is a CUDA graph replayed once per sweep. While profiling is on, a
// second capture of the sweep holds an external event-record node before and
// after each pass and replaces every 16th replay (sweeps 16, 32, ... of each
// run of replays); before each of its replays
// the nodes are pointed at fresh events from a per-device pool. The (start,
// stop) pairs are only queued; nnc_profile_read reads them with
// cudaEventElapsedTime, so timing reads never stall a fit.
#pragma once

#include <vector>

#include "common.cuh"

namespace nnc {

constexpr int kProfileKinds = 6;

struct PassEvents {
  cudaEvent_t start[2];
  cudaEvent_t stop[2];
};

bool profile_enabled();

class PassProfiler {
 public:
  // kind_base: 0 for the SIMT passes (kinds 0, 1), 2 for the BF16
  // tensor-core passes (kinds 2, 3), 4 for the TF32x3 ones (kinds 4, 5).
  explicit PassProfiler(int kind_base = 0) : kind_base_(kind_base) {}
  int init(int launches);                        // reserve 4 events per launch
  const PassEvents* capture_events() const { return &cap_; }
  int bind(cudaGraph_t graph);                   // find the 4 event-record nodes
  int set_launch(cudaGraphExec_t exec, int t);   // point them at launch t's events
  int collect(int launches);                     // queue the pairs for nnc_profile_read

 private:
  int kind_base_;
  int dev_ = 0;
  std::vector<cudaEvent_t> ev_;
  PassEvents cap_{};
  cudaGraphNode_t node_[4] = {};
};

}  // namespace nnc
