// Batched fits of small problems, one block per problem (small_batched.cu).
#pragma once

#include "common.cuh"

namespace nnc {

template <typename T>
int ntd_small_batched(int n_jobs, const ntd_small_job* jobs, int iters, double eps,
                      double* rel_errs, cudaStream_t s);
template <typename T>
int nmf_small_batched(int n_jobs, const nmf_job* jobs, int iters, double eps, double* rel_errs,
                      cudaStream_t s);
template <typename T>
int lifted_small_batched(int n_jobs, const lifted_job* jobs, double* rel_errs, cudaStream_t s);
// nnCP of large 3-way tensors (the tensor stays in global memory, two passes
// over it per sweep), one block per job; r <= 16. Jobs that fail
// nncp_job_valid are skipped (statuses: INVALID_ARG); statuses (device, or
// NULL) gets each fit's NNC_OK / NNC_ERR_NONFINITE as in launch_nncp.
template <typename T>
int nncp_l2_batched(int n_jobs, const nncp_job* jobs, int iters, double eps, double* rel_errs,
                    int* statuses, cudaStream_t s);
// Shared-memory elements one job of nncp_l2_batched needs (a 3-way job).
size_t cpx_l2_elems(const nncp_job& j);

}  // namespace nnc
