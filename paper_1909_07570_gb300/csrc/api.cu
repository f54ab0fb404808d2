// C ABI of the nnCANDELINC library: argument checks and the stream-ordered
// orchestration of the kernels (Alg. 1 of arXiv 1909.07570).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "autotune.cuh"
#include "kernels.cuh"
#include "lifted.cuh"
#include "nncp.cuh"
#include "ntd.cuh"
#include "residual.cuh"
#include "small_batched.cuh"
#include "tc_ttm.cuh"

namespace nnc {

namespace {
thread_local std::string g_detail;
thread_local int g_refine_sweep = -1;  // nnc_last_refine_sweep()
}

void set_error_detail(const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  g_detail = buf;
}

void set_error_detail_text(const std::string& s) { g_detail = s; }

void clear_error_detail() { g_detail.clear(); }

int check_trace_finite(const int* counter, cudaStream_t s, const char* what) {
  int h[2] = {0, 0};
  NNC_CUDA_TRY(cudaMemcpyAsync(h, counter, sizeof(h), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[1] != 0) {
    g_detail = std::string(what) + ": the residual of sweep " + std::to_string(h[1]) +
               " is not finite (an overflow or a NaN during the fit)";
    return NNC_ERR_NONFINITE;
  }
  return NNC_OK;
}

int check_opts(const nnc_opts* o) {
  if (o == nullptr) return NNC_ERR_INVALID_ARG;
  if (o->iters < 0 || !(o->eps > 0.0)) return NNC_ERR_INVALID_ARG;
  if (o->refine_iters < 0 || o->refine_iters > o->iters) return NNC_ERR_INVALID_ARG;
  if (o->exact_every < 0 || !(o->refine_tol >= 0.0) || !std::isfinite(o->refine_tol))
    return NNC_ERR_INVALID_ARG;
  return NNC_OK;
}

namespace {
std::atomic<long long> g_kernel_launches{0};
// Countdown of nnc_debug_fail_alloc: the allocation that takes it from 1 to 0
// fails; 0 means disarmed.
std::atomic<int> g_fail_alloc{0};
}

bool alloc_injection_fires() {
  int v = g_fail_alloc.load(std::memory_order_relaxed);
  while (v > 0) {
    if (g_fail_alloc.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
  }
  return false;
}

void note_launch(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) return;
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

void note_graph_launches(long long kernels) {
  g_kernel_launches.fetch_add(kernels, std::memory_order_relaxed);
}

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, size_t>> set;
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& kv : set) {
    if (kv.first.first == dev && kv.first.second == kernel) {
      if (kv.second >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) kv.second = bytes;
      return e;
    }
  }
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set.push_back({{dev, kernel}, bytes});
  return e;
}

int device_sm_count() {
  static std::atomic<int> cache[64];  // 0 until first read (zero-initialised static)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int c = cache[dev].load(std::memory_order_relaxed);
  if (c == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
    cache[dev].store(n, std::memory_order_relaxed);
    c = n;
  }
  return c;
}

namespace {

int check_shape(int d, const int64_t* dims, const int* m, int max_m) {
  if (dims == nullptr || m == nullptr) return NNC_ERR_INVALID_ARG;
  for (int n = 0; n < d; ++n) {
    if (dims[n] < 1 || dims[n] > (1LL << 31) - 1) return NNC_ERR_INVALID_ARG;
    if (m[n] < 1 || m[n] > max_m) return NNC_ERR_INVALID_ARG;
  }
  return NNC_OK;
}

template <typename T>
int nncp_run(int n_jobs, const nncp_job* jobs, const nnc_opts* o, double* rel_errs, int* statuses,
             cudaStream_t s) {
  NncpRoute rt;
  NNC_TRY(nncp_route<T>(n_jobs, jobs, statuses != nullptr, &rt));
  if (rt.cluster)
    return nncp_cluster_batched<T>(n_jobs, jobs, o->iters, o->eps, rel_errs, statuses, s);
  if (rt.two_pass)
    return nncp_l2_batched<T>(n_jobs, jobs, o->iters, o->eps, rel_errs, statuses, s);
  Scratch sc(s);
  nncp_job* dev = nullptr;
  NNC_TRY(sc.get(&dev, (size_t)n_jobs));
  // A private pageable copy: the runtime stages it before cudaMemcpyAsync
  // returns, so neither buffer has to outlive this call.
  std::vector<nncp_job> host(jobs, jobs + n_jobs);
  NNC_CUDA_TRY(cudaMemcpyAsync(dev, host.data(), sizeof(nncp_job) * n_jobs,
                               cudaMemcpyHostToDevice, s));
  const TuneKey key = nncp_tune_key(jobs, n_jobs, sizeof(T));
  NNC_TRY(run_tuned(key, o->iters, 256, s, [&](int threads, int sweeps, bool last) -> int {
    NNC_CUDA_TRY(launch_nncp<T>(dev, n_jobs, rt.smem, sweeps, o->eps, last ? rel_errs : nullptr,
                                last ? statuses : nullptr, s, threads));
    return NNC_OK;
  }));
  return NNC_OK;
}

// Shared checks of the two lifted-loss entries.
int check_lifted(const void* X, int d, const int64_t* dims, const int* m, int r, const void* F,
                 const void* B) {
  if (X == nullptr || F == nullptr || B == nullptr) return NNC_ERR_INVALID_ARG;
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  if (r < 1 || r > 64) return NNC_ERR_INVALID_ARG;
  return check_shape(d, dims, m, 64);
}

template <typename T>
int lifted_grad_call(const void* X, int d, const int64_t* dims, const int* m, int r, bool tc,
                     const void* const* F, const void* const* B, void* const* gF,
                     void* const* gB, double* loss, cudaStream_t s) {
  T *f[4], *b[4], *gf[4], *gb[4];
  for (int n = 0; n < d; ++n) {
    if (F[n] == nullptr || B[n] == nullptr) return NNC_ERR_INVALID_ARG;
    f[n] = static_cast<T*>(const_cast<void*>(F[n]));
    b[n] = static_cast<T*>(const_cast<void*>(B[n]));
    if (gF) {
      if (gF[n] == nullptr || gB[n] == nullptr) return NNC_ERR_INVALID_ARG;
      gf[n] = static_cast<T*>(gF[n]);
      gb[n] = static_cast<T*>(gB[n]);
    }
  }
  return lifted_grad<T>(static_cast<const T*>(X), d, dims, m, r, tc, f, b, gF ? gf : nullptr,
                        gF ? gb : nullptr, loss, s);
}

template <typename T>
int pg_fit_call(const void* X, int d, const int64_t* dims, const int* m, int r, bool tc,
                int steps, void* const* F, void* const* B, double* trace, double* loss,
                cudaStream_t s) {
  T *f[4], *b[4];
  for (int n = 0; n < d; ++n) {
    if (F[n] == nullptr || B[n] == nullptr) return NNC_ERR_INVALID_ARG;
    f[n] = static_cast<T*>(F[n]);
    b[n] = static_cast<T*>(B[n]);
  }
  return lifted_pg_fit<T>(static_cast<const T*>(X), d, dims, m, r, tc, steps, f, b, trace, loss,
                          s);
}
}  // namespace
}  // namespace nnc

using namespace nnc;

extern "C" {

const char* nnc_status_string(int status) {
  switch (status) {
    case NNC_OK: return "ok";
    case NNC_ERR_INVALID_ARG: return "invalid argument";
    case NNC_ERR_NEGATIVE_INPUT: return "input tensor has a negative entry";
    case NNC_ERR_NONFINITE: return "non-finite value";
    case NNC_ERR_CUDA: return "CUDA error";
    case NNC_ERR_ALLOC: return "scratch allocation failed";
    case NNC_ERR_UNSUPPORTED: return "unsupported by this build";
    case NNC_ERR_TIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

const char* nnc_last_error_detail(void) { return g_detail.c_str(); }

long long nnc_kernel_launches(void) { return g_kernel_launches.load(); }

int nnc_last_refine_sweep(void) { return g_refine_sweep; }

int nnc_debug_fail_alloc(int nth) {
  return g_fail_alloc.exchange(nth > 0 ? nth : 0);
}

int nnc_wait_selftest(long long cycles, void* stream) {
  g_detail.clear();
  return tc::wait_selftest(cycles, static_cast<cudaStream_t>(stream));
}

int nnc_autotune_enable(int on) {
  const bool was = autotune_on();
  autotune_set(on != 0);
  return was ? 1 : 0;
}

int ntd_fit(const void* X, int d, const int64_t* dims, const int* m, int precision,
            const nnc_opts* opts, void* const* F, void* G, double* rel_err_trace,
            double* rel_err, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (X == nullptr || F == nullptr || G == nullptr) return NNC_ERR_INVALID_ARG;
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  NNC_TRY(check_shape(d, dims, m, 64));
  for (int n = 0; n < d; ++n)
    if (F[n] == nullptr) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d == 4) {
    if (opts->exact_every > 0 || opts->refine_tol > 0.0) {
      g_detail = "ntd_fit: exact checkpoints and the refinement trigger serve d = 3 only";
      return NNC_ERR_UNSUPPORTED;
    }
    switch (precision) {
      case NNC_FP64:
        return ntd_fit_nway<double>(static_cast<const double*>(X), 4, dims, m, false,
                                    opts->iters, opts->eps, reinterpret_cast<double* const*>(F),
                                    static_cast<double*>(G), rel_err_trace, rel_err, s);
      case NNC_FP32:
      case NNC_FP32_SIMT:
        return ntd_fit_nway<float>(static_cast<const float*>(X), 4, dims, m,
                                   precision == NNC_FP32, opts->iters, opts->eps,
                                   reinterpret_cast<float* const*>(F), static_cast<float*>(G),
                                   rel_err_trace, rel_err, s);
      case NNC_BF16_REFINE:
        return NNC_ERR_UNSUPPORTED;
      default:
        return NNC_ERR_INVALID_ARG;
    }
  }
  switch (precision) {
    case NNC_FP64:
      return ntd_fit3<double>(static_cast<const double*>(X), dims, m, opts,
                              reinterpret_cast<double* const*>(F), static_cast<double*>(G),
                              rel_err_trace, rel_err, false, s);
    case NNC_FP32:
    case NNC_FP32_SIMT:
      return ntd_fit3<float>(static_cast<const float*>(X), dims, m, opts,
                             reinterpret_cast<float* const*>(F), static_cast<float*>(G),
                             rel_err_trace, rel_err, precision == NNC_FP32, s);
    case NNC_BF16_REFINE: {
      int from = -1;
      const int st = ntd_fit3_bf16(static_cast<const float*>(X), dims, m, opts,
                                   reinterpret_cast<float* const*>(F), static_cast<float*>(G),
                                   rel_err_trace, rel_err, &from, s);
      g_refine_sweep = from;
      return st;
    }
    default:
      return NNC_ERR_INVALID_ARG;
  }
}

int ntd_fit_batched(int n_jobs, const ntd_job* jobs, int precision, const nnc_opts* opts,
                    int concurrency, double* rel_errs, int* statuses, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return NNC_ERR_INVALID_ARG;
  if (n_jobs == 0) return NNC_OK;
  int workers = concurrency <= 0 ? 8 : (concurrency > 32 ? 32 : concurrency);
  if (workers > n_jobs) workers = n_jobs;
  int dev = 0;
  NNC_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t fork = nullptr;
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventRecord(fork, s));
  std::vector<int> st(n_jobs, NNC_OK);
  std::vector<double> errs(n_jobs, 0.0);
  std::vector<std::string> detail(n_jobs);
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  pool.reserve(workers);
  for (int w = 0; w < workers; ++w) {
    pool.emplace_back([&]() {
      cudaStream_t ws = nullptr;
      if (cudaSetDevice(dev) != cudaSuccess ||
          cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(ws, fork, 0) != cudaSuccess) {
        for (int j = next.fetch_add(1); j < n_jobs; j = next.fetch_add(1)) st[j] = NNC_ERR_CUDA;
        if (ws) cudaStreamDestroy(ws);
        return;
      }
      for (int j = next.fetch_add(1); j < n_jobs; j = next.fetch_add(1)) {
        const ntd_job& jb = jobs[j];
        st[j] = ntd_fit(jb.X, jb.d, jb.dims, jb.m, precision, opts, jb.F, jb.G, jb.trace,
                        &errs[j], ws);
        if (st[j] != NNC_OK) detail[j] = nnc_last_error_detail();
      }
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
    });
  }
  for (auto& t : pool) t.join();
  cudaEventDestroy(fork);
  int first = NNC_OK;
  for (int j = 0; j < n_jobs; ++j) {
    if (statuses) statuses[j] = st[j];
    if (rel_errs) rel_errs[j] = st[j] == NNC_OK ? errs[j] : NAN;
    if (st[j] != NNC_OK && first == NNC_OK) {
      first = st[j];
      g_detail = "job " + std::to_string(j) + ": " + detail[j];
    }
  }
  return first;
}

int ntd_fit_small_batched(int n_jobs, const ntd_small_job* jobs, int precision,
                          const nnc_opts* opts, double* rel_errs, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return NNC_ERR_INVALID_ARG;
  if (n_jobs == 0) return NNC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64)
    return ntd_small_batched<double>(n_jobs, jobs, opts->iters, opts->eps, rel_errs, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return ntd_small_batched<float>(n_jobs, jobs, opts->iters, opts->eps, rel_errs, s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int nmf_fit_batched(int n_jobs, const nmf_job* jobs, int precision, const nnc_opts* opts,
                    double* rel_errs, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return NNC_ERR_INVALID_ARG;
  if (n_jobs == 0) return NNC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64)
    return nmf_small_batched<double>(n_jobs, jobs, opts->iters, opts->eps, rel_errs, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return nmf_small_batched<float>(n_jobs, jobs, opts->iters, opts->eps, rel_errs, s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int lifted_rel_err_batched(int n_jobs, const lifted_job* jobs, int precision, double* rel_errs,
                           void* stream) {
  g_detail.clear();
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return NNC_ERR_INVALID_ARG;
  if (n_jobs == 0) return NNC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64) return lifted_small_batched<double>(n_jobs, jobs, rel_errs, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return lifted_small_batched<float>(n_jobs, jobs, rel_errs, s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int nncp_core_fit(const void* G, int d, const int* m, int r, int precision, const nnc_opts* opts,
                  void* const* B, double* rel_err, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (G == nullptr || B == nullptr || m == nullptr || (d != 3 && d != 4)) return NNC_ERR_INVALID_ARG;
  nncp_job job;
  memset(&job, 0, sizeof(job));
  job.G = G;
  job.d = d;
  job.r = r;
  for (int k = 0; k < d; ++k) {
    job.m[k] = m[k];
    job.B[k] = B[k];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc(s);
  double* dev_err = nullptr;
  if (rel_err) NNC_TRY(sc.get(&dev_err, 1));
  int st;
  if (precision == NNC_FP64)
    st = nncp_run<double>(1, &job, opts, dev_err, nullptr, s);
  else if (precision == NNC_FP32 || precision == NNC_BF16_REFINE || precision == NNC_FP32_SIMT)
    st = nncp_run<float>(1, &job, opts, dev_err, nullptr, s);
  else
    return NNC_ERR_INVALID_ARG;
  if (st != NNC_OK) return st;
  if (rel_err) {
    NNC_CUDA_TRY(cudaMemcpyAsync(rel_err, dev_err, sizeof(double), cudaMemcpyDeviceToHost, s));
    NNC_CUDA_TRY(cudaStreamSynchronize(s));
    if (!std::isfinite(*rel_err)) {
      set_error_detail_text("nncp_core_fit: the fit's residual is not finite");
      return NNC_ERR_NONFINITE;
    }
  }
  return NNC_OK;
}

int nncp_core_fit_batched(int n_jobs, const nncp_job* jobs, int precision, const nnc_opts* opts,
                          double* rel_errs, int* statuses, void* stream) {
  g_detail.clear();
  NNC_TRY(check_opts(opts));
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return NNC_ERR_INVALID_ARG;
  if (n_jobs == 0) return NNC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64) return nncp_run<double>(n_jobs, jobs, opts, rel_errs, statuses, s);
  if (precision == NNC_FP32 || precision == NNC_BF16_REFINE || precision == NNC_FP32_SIMT)
    return nncp_run<float>(n_jobs, jobs, opts, rel_errs, statuses, s);
  return NNC_ERR_INVALID_ARG;
}

int nnc_mode_product(const void* X, int d, const int64_t* dims, int mode, const void* F, int Q,
                     int precision, void* out, void* stream) {
  g_detail.clear();
  if (X == nullptr || F == nullptr || out == nullptr || dims == nullptr) return NNC_ERR_INVALID_ARG;
  if (d != 3 || mode < 0 || mode > 2 || Q < 1 || Q > 64) return NNC_ERR_INVALID_ARG;
  for (int n = 0; n < 3; ++n)
    if (dims[n] < 1 || dims[n] > (1LL << 31) - 1) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t L = 1, C = 1;
  for (int n = 0; n < mode; ++n) L *= dims[n];
  for (int n = mode + 1; n < 3; ++n) C *= dims[n];
  const int J = static_cast<int>(dims[mode]);
  Scratch sc(s);
  if (precision == NNC_BF16_REFINE || (precision == NNC_FP32 && mode != 1)) {
    if (mode == 1) return NNC_ERR_UNSUPPORTED;
    tc::TcPlan plan;
    const int kind = precision == NNC_BF16_REFINE ? tc::kKindBf16 : tc::kKindTf32x3;
    const int st = plan.init(kind, static_cast<const float*>(X), dims[0], dims[1], dims[2], Q, Q,
                             sc, s);
    if (st == NNC_OK) {
      if (mode == 2)
        NNC_TRY(plan.pass3(static_cast<const float*>(F), static_cast<float*>(out), s));
      else
        NNC_TRY(plan.pass1(static_cast<const float*>(F), static_cast<float*>(out), s));
      return plan.check(s);
    }
    if (st != NNC_ERR_UNSUPPORTED || precision == NNC_BF16_REFINE) return st;
    // TF32x3 cannot take this shape: FP32 SIMT below.
  }
  const size_t cap = static_cast<size_t>(L * Q * C) * 8;
  if (precision == NNC_FP64) {
    double* split = nullptr;
    NNC_TRY(sc.get(&split, cap));
    NNC_CUDA_TRY(launch_ttm<double>(static_cast<const double*>(X), L, J, C,
                                    static_cast<const double*>(F), Q, 1, Q,
                                    static_cast<double*>(out), split, cap, s));
  } else if (precision == NNC_FP32 || precision == NNC_FP32_SIMT) {
    float* split = nullptr;
    NNC_TRY(sc.get(&split, cap));
    // NNC_FP32, mode 1: the column product on the tensor cores where it applies.
    auto ttm = precision == NNC_FP32 ? launch_ttm_tc<float> : launch_ttm<float>;
    NNC_CUDA_TRY(ttm(static_cast<const float*>(X), L, J, C, static_cast<const float*>(F), Q, 1, Q,
                     static_cast<float*>(out), split, cap, s));
  } else {
    return NNC_ERR_INVALID_ARG;
  }
  return NNC_OK;
}

int candelinc_lift(int d, const int64_t* dims, const int* m, int r, int precision,
                   const void* const* F, const void* const* B, void* const* A, void* stream) {
  g_detail.clear();
  if (d < 1 || d > 8 || F == nullptr || B == nullptr || A == nullptr || r < 1)
    return NNC_ERR_INVALID_ARG;
  NNC_TRY(check_shape(d, dims, m, 1 << 20));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int n = 0; n < d; ++n) {
    if (F[n] == nullptr || B[n] == nullptr || A[n] == nullptr) return NNC_ERR_INVALID_ARG;
    if (precision == NNC_FP64) {
      NNC_CUDA_TRY(launch_lift<double>(static_cast<const double*>(F[n]),
                                       static_cast<const double*>(B[n]), dims[n], m[n], r,
                                       static_cast<double*>(A[n]), s));
    } else if (precision == NNC_FP32 || precision == NNC_BF16_REFINE ||
               precision == NNC_FP32_SIMT) {
      NNC_CUDA_TRY(launch_lift<float>(static_cast<const float*>(F[n]),
                                      static_cast<const float*>(B[n]), dims[n], m[n], r,
                                      static_cast<float*>(A[n]), s));
    } else {
      return NNC_ERR_INVALID_ARG;
    }
  }
  return NNC_OK;
}

int candelinc_lifted_grad(const void* X, int d, const int64_t* dims, const int* m, int r,
                          int precision, const void* const* F, const void* const* B,
                          void* const* gF, void* const* gB, double* loss, void* stream) {
  g_detail.clear();
  NNC_TRY(check_lifted(X, d, dims, m, r, F, B));
  if ((gF == nullptr) != (gB == nullptr)) return NNC_ERR_INVALID_ARG;
  if (gF == nullptr && loss == nullptr) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64)
    return lifted_grad_call<double>(X, d, dims, m, r, false, F, B, gF, gB, loss, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return lifted_grad_call<float>(X, d, dims, m, r, precision == NNC_FP32, F, B, gF, gB, loss,
                                   s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int candelinc_pg_fit(const void* X, int d, const int64_t* dims, const int* m, int r,
                     int precision, int steps, void* const* F, void* const* B, double* trace,
                     double* loss, void* stream) {
  g_detail.clear();
  NNC_TRY(check_lifted(X, d, dims, m, r, F, B));
  if (steps < 0) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64)
    return pg_fit_call<double>(X, d, dims, m, r, false, steps, F, B, trace, loss, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return pg_fit_call<float>(X, d, dims, m, r, precision == NNC_FP32, steps, F, B, trace, loss,
                              s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int nncp_tensor_fit(const void* X, int d, const int64_t* dims, int r, int precision,
                    const nnc_opts* opts, void* const* A, double* trace, double* rel_err,
                    void* stream) {
  g_detail.clear();
  if (X == nullptr || A == nullptr) return NNC_ERR_INVALID_ARG;
  NNC_TRY(check_opts(opts));
  if ((d != 3 && d != 4) || r < 1 || r > 64) return NNC_ERR_INVALID_ARG;
  int m[4] = {r, r, r, r};
  NNC_TRY(check_shape(d, dims, m, 64));
  for (int n = 0; n < d; ++n)
    if (A[n] == nullptr) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64) {
    double* a[4];
    for (int n = 0; n < d; ++n) a[n] = static_cast<double*>(A[n]);
    return nncp_tensor_fit<double>(static_cast<const double*>(X), d, dims, r, false, opts->iters,
                                   opts->eps, opts->exact_every, a, trace, rel_err, s);
  }
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT) {
    float* a[4];
    for (int n = 0; n < d; ++n) a[n] = static_cast<float*>(A[n]);
    return nncp_tensor_fit<float>(static_cast<const float*>(X), d, dims, r,
                                  precision == NNC_FP32, opts->iters, opts->eps,
                                  opts->exact_every, a, trace, rel_err, s);
  }
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int nmf_fit(const void* A, int64_t N, int r, int m, int precision, const nnc_opts* opts, void* F,
            void* B, double* trace, double* rel_err, void* stream) {
  g_detail.clear();
  if (A == nullptr || F == nullptr || B == nullptr || opts == nullptr || opts->iters < 0 ||
      !(opts->eps > 0.0))
    return NNC_ERR_INVALID_ARG;
  if (N < 1 || N > (1LL << 31) - 1 || r < 1 || r > 1024 || m < 1 || m > 1024)
    return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == NNC_FP64)
    return nmf_fit<double>(static_cast<const double*>(A), N, r, m, opts->iters, opts->eps,
                           static_cast<double*>(F), static_cast<double*>(B), trace, rel_err, s);
  if (precision == NNC_FP32 || precision == NNC_FP32_SIMT)
    return nmf_fit<float>(static_cast<const float*>(A), N, r, m, opts->iters, opts->eps,
                          static_cast<float*>(F), static_cast<float*>(B), trace, rel_err, s);
  return precision == NNC_BF16_REFINE ? NNC_ERR_UNSUPPORTED : NNC_ERR_INVALID_ARG;
}

int candelinc_alg2(const void* X, int d, const int64_t* dims, const int* m, int r, int precision,
                   const nnc_opts* cp_opts, const nnc_opts* nmf_opts, void* const* A,
                   void* const* F, void* const* B, double* cp_rel_err, double* nmf_rel_errs,
                   void* stream) {
  g_detail.clear();
  if (F == nullptr || B == nullptr || m == nullptr) return NNC_ERR_INVALID_ARG;
  NNC_TRY(nncp_tensor_fit(X, d, dims, r, precision, cp_opts, A, nullptr, cp_rel_err, stream));
  for (int n = 0; n < d; ++n) {
    if (m[n] < 1 || m[n] > 1024) return NNC_ERR_INVALID_ARG;
    NNC_TRY(nmf_fit(A[n], dims[n], r, m[n], precision, nmf_opts, F[n], B[n], nullptr,
                    nmf_rel_errs ? nmf_rel_errs + n : nullptr, stream));
  }
  return NNC_OK;
}

int recon_residual(const void* X, int d, const int64_t* dims, int precision, int model,
                   const int* m, int r, const void* const* factors, const void* G,
                   double* resid_norm, double* x_norm, void* stream) {
  g_detail.clear();
  if (X == nullptr || factors == nullptr || dims == nullptr) return NNC_ERR_INVALID_ARG;
  if (model != 0 && model != 1) return NNC_ERR_INVALID_ARG;
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  for (int n = 0; n < d; ++n) {
    if (dims[n] < 1 || factors[n] == nullptr) return NNC_ERR_INVALID_ARG;
    if (model == 0 && (m == nullptr || m[n] < 1 || m[n] > 64)) return NNC_ERR_INVALID_ARG;
  }
  if (model == 0 && G == nullptr) return NNC_ERR_INVALID_ARG;
  if (model == 1 && (r < 1 || r > 64)) return NNC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch sc(s);
  double* out2 = nullptr;
  NNC_TRY(sc.get(&out2, 2));
  if (precision == NNC_FP64) {
    NNC_TRY(residual_device<double>(static_cast<const double*>(X), d, dims, model, m, r,
                                     reinterpret_cast<const double* const*>(factors),
                                     static_cast<const double*>(G), out2, sc, s));
  } else if (precision == NNC_FP32 || precision == NNC_BF16_REFINE ||
             precision == NNC_FP32_SIMT) {
    NNC_TRY(residual_device<float>(static_cast<const float*>(X), d, dims, model, m, r,
                                    reinterpret_cast<const float* const*>(factors),
                                    static_cast<const float*>(G), out2, sc, s));
  } else {
    return NNC_ERR_INVALID_ARG;
  }
  double h[2];
  NNC_CUDA_TRY(cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (resid_norm) *resid_norm = sqrt(h[0]);
  if (x_norm) *x_norm = sqrt(h[1]);
  return NNC_OK;
}

}  // extern "C"
