// Launcher of the core nnCPD kernel (nncp.cu).
#pragma once

#include "common.cuh"

namespace nnc {

// Dynamic shared memory one block needs for job `j` with elements of `elem` bytes.
size_t nncp_smem_bytes(const nncp_job& j, size_t elem);

// One block per job; jobs_dev is a device array of n_jobs descriptors whose
// cores and factors hold elements of type T. rel_errs (device, n_jobs) may be
// NULL.
template <typename T>
cudaError_t launch_nncp(const nncp_job* jobs_dev, int n_jobs, size_t smem, int iters, double eps,
                        double* rel_errs, cudaStream_t s);

}  // namespace nnc
