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
// over it per sweep), one block per job; r <= 16.
template <typename T>
int nncp_l2_batched(int n_jobs, const nncp_job* jobs, int iters, double eps, double* rel_errs,
                    cudaStream_t s);
// Whether nncp_l2_batched can take the batch (every job 3-way, r <= 16, its
// arrays within one block's shared memory).
template <typename T>
bool nncp_l2_fits(int n_jobs, const nncp_job* jobs);

}  // namespace nnc
