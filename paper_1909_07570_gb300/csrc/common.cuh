// Shared host/device helpers of the nnCANDELINC CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nncandelinc.h"

namespace nnc {

// Records the text of a failed CUDA call for nnc_last_error_detail().
void set_error_detail(const char* what, cudaError_t e);
void set_error_detail_text(const std::string& s);

#define NNC_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) {                               \
      ::nnc::set_error_detail(#expr, e__);                  \
      return NNC_ERR_CUDA;                                  \
    }                                                       \
  } while (0)

#define NNC_TRY(expr)                                       \
  do {                                                      \
    int st__ = (expr);                                      \
    if (st__ != NNC_OK) return st__;                        \
  } while (0)

// True when the test hook nnc_debug_fail_alloc has armed a failure for this
// allocation (host-side failure injection; off unless a caller arms it).
bool alloc_injection_fires();

// Stream-ordered scratch: every block is taken with cudaMallocAsync on the
// call's stream and returned with cudaFreeAsync when the arena dies.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : stream_(s) {}
  ~Scratch() { release(); }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;

  template <typename T>
  int get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    if (alloc_injection_fires()) {
      set_error_detail_text("scratch allocation failed (injected by nnc_debug_fail_alloc)");
      return NNC_ERR_ALLOC;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), stream_);
    if (e != cudaSuccess) {
      set_error_detail("cudaMallocAsync", e);
      (void)cudaGetLastError();
      return NNC_ERR_ALLOC;
    }
    if (n_ == kMax) {
      cudaFreeAsync(p, stream_);
      set_error_detail_text("scratch arena: too many blocks");
      return NNC_ERR_ALLOC;
    }
    blocks_[n_++] = p;
    *out = static_cast<T*>(p);
    return NNC_OK;
  }

  void release() {
    for (int i = n_ - 1; i >= 0; --i) cudaFreeAsync(blocks_[i], stream_);
    n_ = 0;
  }

 private:
  static constexpr int kMax = 64;
  cudaStream_t stream_;
  void* blocks_[kMax] = {};
  int n_ = 0;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Dynamic shared memory the one-block-per-job kernels may ask for.
constexpr size_t kSmemBudget = 200 * 1024;

// Clears this thread's error detail (every ABI call does so on entry).
void clear_error_detail();

// Checks an nnc_opts: iters >= 0, eps > 0, 0 <= refine_iters <= iters.
int check_opts(const nnc_opts* o);

// NNC_ERR_NONFINITE (with a detail naming `what` and the first bad sweep) when
// the trace counter pair of a fit (see trace_record) saw a non-finite entry;
// synchronises `s`.
int check_trace_finite(const int* counter, cudaStream_t s, const char* what);

int device_sm_count();

// Raises `kernel`'s dynamic shared-memory limit on the current device to at
// least `bytes` and never lowers it: a launch captured into a graph keeps the
// size it was captured with while later launches of the same kernel may ask
// for less.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);

// Counts one kernel launch of this library (nnc_kernel_launches). Launches
// made while `s` is being captured into a graph are counted when the graph is
// replayed instead (note_graph_launches).
void note_launch(cudaStream_t s);
void note_graph_launches(long long kernels);

// Programmatic dependent launch. A kernel launched this way may be scheduled
// while the kernel before it on the stream is still running; it must call
// pdl_wait() before touching global memory that kernel writes (or reads and
// this one writes), and at least one of its threads must call it, so that its
// own completion still implies the completion of every kernel before it.
// Without a programmatic predecessor pdl_wait() returns at once.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// Waits until the programmatic predecessor grid has completed and its memory
// operations are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the programmatic successor grid be scheduled before this one ends.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One entry of a fit's per-sweep trace. `counter` points at two ints that the
// fit clears before its first sweep: counter[0] counts the entries recorded,
// counter[1] stays 0 until an entry (or a sum it was formed from) is not
// finite and then holds the 1-based index of the first such sweep. The value
// goes to trace[counter[0] * stride] when a trace is kept. One thread calls it.
__device__ __forceinline__ void trace_record(int* counter, double* trace, int stride, double value,
                                             bool finite) {
  const int t = counter[0];
  if (trace) trace[(int64_t)t * stride] = value;
  if (!(finite && isfinite(value)) && counter[1] == 0) counter[1] = t + 1;
  counter[0] = t + 1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread gets the result. `sh` holds >= 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  T t = (threadIdx.x < nwarps) ? sh[threadIdx.x] : T(0);
  if (warp == 0) {
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// Two FP64 sums over e < n, sum_e f(e).x and sum_e f(e).y, in an order fixed by
// n alone (not by the block size): virtual lane v < kFixedLanes adds the terms
// e = v, v + kFixedLanes, ... in order, then a fixed tree adds the lanes. `part`
// is 2 kFixedLanes doubles of shared memory. Every thread gets both sums.
constexpr int kFixedLanes = 256;
template <typename F>
__device__ double2 fixed_sums2(int64_t n, F f, double* part) {
  for (int v = threadIdx.x; v < kFixedLanes; v += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int64_t e = v; e < n; e += kFixedLanes) {
      const double2 t = f(e);
      a += t.x;
      b += t.y;
    }
    part[v] = a;
    part[kFixedLanes + v] = b;
  }
  __syncthreads();
  for (int h = kFixedLanes / 2; h > 0; h >>= 1) {
    for (int v = threadIdx.x; v < h; v += blockDim.x) {
      part[v] += part[v + h];
      part[kFixedLanes + v] += part[kFixedLanes + v + h];
    }
    __syncthreads();
  }
  const double2 r = make_double2(part[0], part[kFixedLanes]);
  __syncthreads();
  return r;
}

// ---- cp.async staging (element granularity, zero fill outside the range) ----
template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 16-byte cp.async of one vector (16 / sizeof(T) elements); the first `valid`
// elements are copied, the rest of the vector is zero.
template <typename T>
__device__ __forceinline__ void cp_vec(T* dst, const T* src, int valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int n = valid * (int)sizeof(T);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n)
               : "memory");
}

}  // namespace nnc
