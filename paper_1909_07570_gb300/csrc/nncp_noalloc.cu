// nncp_core_fit_batched_noalloc: the batched core nnCPD for callers that must
// not allocate device memory.
//
// nncp_core_fit_batched takes its job table (one descriptor per fit) from
// cudaMallocAsync. Some callers cannot let a library allocate: a host runtime
// that owns all device memory through its own pool or arena and forbids
// allocations behind its back, a real-time or latency-critical loop where an
// allocation may stall or fail under memory pressure, or a process that has
// handed nearly all of the GPU's memory to a framework cache. This entry point
// runs the one-pass core kernel with the job table in a fixed array in the
// library's own device memory instead, so the call allocates nothing. Batches
// that the allocating call would send to its two-pass kernel (which takes its
// own table from the allocator) are refused, so every batch this call accepts
// runs exactly the kernel, launch shape and sums of the allocating call.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocMaxJobs descriptors, 256 KiB) until the process
// exits. Host code may not use its name as a device address, so the address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on it.
#include <cstdio>
#include <mutex>

#include "nncp.cuh"

namespace nnc {
namespace {

constexpr int kNoAllocMaxJobs = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_job_table[kNoAllocMaxJobs * sizeof(nncp_job)];

std::mutex g_table_mu;
void* g_table_addr[kMaxDevices] = {};

// Device address of g_job_table on the current device (set up on first use).
int job_table_address(nncp_job** out) {
  int dev = 0;
  NNC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_detail_text("nncp_core_fit_batched_noalloc: device ordinal out of range");
    return NNC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_table_mu);
  if (g_table_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_job_table);
    if (e != cudaSuccess || p == nullptr) {
      set_error_detail("cudaGetSymbolAddress(job table)", e);
      return NNC_ERR_CUDA;
    }
    g_table_addr[dev] = p;
  }
  *out = static_cast<nncp_job*>(g_table_addr[dev]);
  return NNC_OK;
}

template <typename T>
int run_noalloc(int n_jobs, const nncp_job* jobs, const nnc_opts* o, double* rel_errs,
                int* statuses, cudaStream_t s) {
  // The routing of the allocating call, to the letter (nncp_route).
  NncpRoute rt;
  NNC_TRY(nncp_route<T>(n_jobs, jobs, statuses != nullptr, &rt));
  if (rt.two_pass) {
    set_error_detail_text(
        "nncp_core_fit_batched_noalloc: this batch needs the two-pass kernel (a tensor of 16384 "
        "entries or more, or state beyond one block), which allocates; use "
        "nncp_core_fit_batched");
    return NNC_ERR_UNSUPPORTED;
  }
  nncp_job* table = nullptr;
  NNC_TRY(job_table_address(&table));
  NNC_CUDA_TRY(cudaMemcpyAsync(table, jobs, sizeof(nncp_job) * (size_t)n_jobs,
                               cudaMemcpyHostToDevice, s));
  // A block size tuned by an earlier allocating call of the same class is
  // reused; this call never times anything.
  const int threads = tuned_threads(nncp_tune_key(jobs, n_jobs, sizeof(T)), 256);
  NNC_CUDA_TRY(launch_nncp<T>(table, n_jobs, rt.smem, o->iters, o->eps, rel_errs, statuses, s,
                              threads));
  return NNC_OK;
}

}  // namespace
}  // namespace nnc

using namespace nnc;

extern "C" int nncp_core_fit_batched_noalloc(int n_jobs, const nncp_job* jobs, int precision,
                                             const nnc_opts* opts, double* rel_errs,
                                             int* statuses, void* stream) {
  clear_error_detail();
  if (check_opts(opts) != NNC_OK) {
    set_error_detail_text("nncp_core_fit_batched_noalloc: bad options (iters, refine_iters, eps)");
    return NNC_ERR_INVALID_ARG;
  }
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) {
    set_error_detail_text("nncp_core_fit_batched_noalloc: bad job count or NULL job array");
    return NNC_ERR_INVALID_ARG;
  }
  if (n_jobs > kNoAllocMaxJobs) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "nncp_core_fit_batched_noalloc: %d jobs exceed the fixed table of %d jobs", n_jobs,
             kNoAllocMaxJobs);
    set_error_detail_text(buf);
    return NNC_ERR_INVALID_ARG;
  }
  if (n_jobs == 0) return NNC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64) return run_noalloc<double>(n_jobs, jobs, opts, rel_errs, statuses, s);
  if (precision == NNC_FP32 || precision == NNC_BF16_REFINE || precision == NNC_FP32_SIMT)
    return run_noalloc<float>(n_jobs, jobs, opts, rel_errs, statuses, s);
  set_error_detail_text("nncp_core_fit_batched_noalloc: unknown precision");
  return NNC_ERR_INVALID_ARG;
}
