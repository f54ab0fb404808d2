// Launcher and batch routing of the core nnCPD kernels (nncp.cu).
#pragma once

#include "autotune.cuh"
#include "common.cuh"

namespace nnc {

// Whether one job descriptor is one the batched core fits take: d = 3 or 4,
// 1 <= r <= 32, 1 <= m[n] <= 64, G and every B[n] non-null. The host (when it
// routes a batch) and the kernels (which skip an invalid job and report it in
// its status) apply the same test.
__host__ __device__ inline bool nncp_job_valid(const nncp_job& j) {
  if (j.G == nullptr || (j.d != 3 && j.d != 4) || j.r < 1 || j.r > 32) return false;
  for (int k = 0; k < j.d; ++k)
    if (j.m[k] < 1 || j.m[k] > 64 || j.B[k] == nullptr) return false;
  return true;
}

// Dynamic shared memory one block of the one-pass kernel needs for job `j`
// with elements of `elem` bytes.
size_t nncp_smem_bytes(const nncp_job& j, size_t elem);

// How a batch of core fits runs. Both entry points of the batched fit
// (nncp_core_fit_batched and its no-alloc variant) take their decision here,
// so they cannot drift apart.
struct NncpRoute {
  size_t smem = 0;        // one-pass kernel: dynamic shared memory (largest valid job)
  bool two_pass = false;  // the two-pass sweep (two passes over the tensor) takes the batch
  bool cluster = false;   // ... as one thread-block cluster per fit (nncp_cluster_batched)
  int invalid = 0;        // jobs that fail nncp_job_valid
};

// Routes the valid jobs of a batch with elements of type T. The one-pass
// kernel reads the tensor through L1 once per numerator entry (r times per
// mode and sweep), so a batch holding a tensor of 16384 entries or more goes
// to the two-pass kernel when that kernel can take it (every valid job 3-way,
// r <= 16, its arrays within one block), and so does a batch whose one-pass
// state exceeds 200 KiB of shared memory. UNSUPPORTED (with a detail) when
// neither kernel takes the batch. A two-pass batch runs one cluster of
// cpx_cluster_ctas() CTAs per fit when the clusters of all its valid jobs fit
// on the GPU at once and every job's slabs fit in a CTA's shared memory (a
// few large fits, as in Alg. 1's core fit), else one block per fit. With
// skip_invalid false an invalid job makes the call INVALID_ARG (the detail
// names the job); with it true the invalid jobs are only counted.
template <typename T>
int nncp_route(int n_jobs, const nncp_job* jobs, bool skip_invalid, NncpRoute* rt);

// One block of `threads` threads (32 .. 256) per job; jobs_dev is a device
// array of n_jobs descriptors whose cores and factors hold elements of type T.
// rel_errs (device, n_jobs) may be NULL. statuses (device, n_jobs) may be
// NULL; a block writes NNC_OK, NNC_ERR_NONFINITE (a non-finite entry in its
// fitted factors or in its residual sums, e.g. from a NaN in the core) or
// NNC_ERR_INVALID_ARG (descriptor fails nncp_job_valid: nothing else done).
// Results do not depend on `threads`.
template <typename T>
cudaError_t launch_nncp(const nncp_job* jobs_dev, int n_jobs, size_t smem, int iters, double eps,
                        double* rel_errs, int* statuses, cudaStream_t s, int threads = 256);

// The two-pass sweep with one thread-block cluster per fit (nncp_cluster.cu):
// 3-way jobs, any r <= 32; jobs that fail nncp_job_valid are skipped
// (statuses: INVALID_ARG); statuses and rel_errs as in nncp_l2_batched.
template <typename T>
int nncp_cluster_batched(int n_jobs, const nncp_job* jobs, int iters, double eps,
                         double* rel_errs, int* statuses, cudaStream_t s);
// Shared-memory elements of one CTA of a cluster fit of job j, and the CTAs
// of a cluster.
size_t cpx_cluster_elems(const nncp_job& j);
int cpx_cluster_ctas();

// The tuning class of a batch (largest per-sweep work over the valid jobs,
// number of jobs).
TuneKey nncp_tune_key(const nncp_job* jobs, int n_jobs, size_t elem);

}  // namespace nnc
