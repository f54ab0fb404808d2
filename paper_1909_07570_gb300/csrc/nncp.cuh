// Launcher of the core nnCPD kernel (nncp.cu).
#pragma once

#include "autotune.cuh"
#include "common.cuh"

namespace nnc {

// Dynamic shared memory one block needs for job `j` with elements of `elem` bytes.
size_t nncp_smem_bytes(const nncp_job& j, size_t elem);

// One block of `threads` threads (32 .. 256) per job; jobs_dev is a device
// array of n_jobs descriptors whose cores and factors hold elements of type T.
// rel_errs (device, n_jobs) may be NULL. Results do not depend on `threads`.
template <typename T>
cudaError_t launch_nncp(const nncp_job* jobs_dev, int n_jobs, size_t smem, int iters, double eps,
                        double* rel_errs, cudaStream_t s, int threads = 256);

// The tuning class of a batch (largest per-sweep work, number of jobs).
TuneKey nncp_tune_key(const nncp_job* jobs, int n_jobs, size_t elem);

}  // namespace nnc
