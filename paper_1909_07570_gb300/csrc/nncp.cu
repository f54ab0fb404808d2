// nnCPD of Tucker cores (Alg. 1, step 2): multiplicative updates of
// B^(1), ..., B^(d) for 1/2 ||G - I x_n B^(n)||_F^2, one thread block per fit.
//
// A block keeps every B^(k) (m_k x r) and its Gram B^(k)T B^(k) (r x r) in
// shared memory and reads the core G through L1. A sweep, for n = 1..d:
//   V   = Hadamard product over k != n of Gram_k
//   Num = unfold_n(G) KR_{k!=n} B^(k)   (MTTKRP, factored loop over the modes)
//   B^(n) <- max(B^(n) * Num / max(B^(n) V, eps), 0);  Gram_n <- B^(n)T B^(n)
// The same kernel serves one fit (nncp_core_fit) and many uneven fits in one
// launch (nncp_core_fit_batched); no block waits on another.
#include <string>

#include "kernels.cuh"
#include "nncp.cuh"
#include "small_batched.cuh"

namespace nnc {
namespace {

constexpr int kThreads = 256;

template <typename T, int D>
__device__ T mttkrp_entry(const T* __restrict__ G, const int* m, const int64_t* st,
                          T* const* Bs, int r, int n, int i, int q) {
  int o[D - 1];
  {
    int t = 0;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k != n) o[t++] = k;
  }
  const T* g0 = G + (int64_t)i * st[n];
  T s = T(0);
  if constexpr (D == 3) {
    for (int j0 = 0; j0 < m[o[0]]; ++j0) {
      const T* g1 = g0 + j0 * st[o[0]];
      T inner = T(0);
      for (int j1 = 0; j1 < m[o[1]]; ++j1)
        inner = fma(g1[j1 * st[o[1]]], Bs[o[1]][j1 * r + q], inner);
      s = fma(Bs[o[0]][j0 * r + q], inner, s);
    }
  } else {
    for (int j0 = 0; j0 < m[o[0]]; ++j0) {
      const T* g1 = g0 + j0 * st[o[0]];
      T mid = T(0);
      for (int j1 = 0; j1 < m[o[1]]; ++j1) {
        const T* g2 = g1 + j1 * st[o[1]];
        T inner = T(0);
        for (int j2 = 0; j2 < m[o[2]]; ++j2)
          inner = fma(g2[j2 * st[o[2]]], Bs[o[2]][j2 * r + q], inner);
        mid = fma(Bs[o[1]][j1 * r + q], inner, mid);
      }
      s = fma(Bs[o[0]][j0 * r + q], mid, s);
    }
  }
  return s;
}

template <typename T, int D>
__device__ void fit_one(const nncp_job& job, int iters, T eps, unsigned char* smem,
                        double* rel_err_out, int* status_out) {
  const int r = job.r;
  int m[D];
  int64_t st[D];
#pragma unroll
  for (int k = 0; k < D; ++k) m[k] = job.m[k];
  st[D - 1] = 1;
#pragma unroll
  for (int k = D - 2; k >= 0; --k) st[k] = st[k + 1] * m[k + 1];
  int mmax = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) mmax = m[k] > mmax ? m[k] : mmax;

  // Shared memory: B^(k) | Gram_k | V | Num
  T* p = reinterpret_cast<T*>(smem);
  T* Bs[D];
  T* Gram[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    Bs[k] = p;
    p += m[k] * r;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    Gram[k] = p;
    p += r * r;
  }
  T* V = p;
  p += r * r;
  T* Num = p;

  const T* G = static_cast<const T*>(job.G);
  const int tid = threadIdx.x;

#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T* src = static_cast<const T*>(job.B[k]);
    for (int e = tid; e < m[k] * r; e += blockDim.x) Bs[k][e] = src[e];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < D; ++k)
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int a = e / r, b = e % r;
      T s = T(0);
      for (int i = 0; i < m[k]; ++i) s = fma(Bs[k][i * r + a], Bs[k][i * r + b], s);
      Gram[k][e] = s;
    }
  __syncthreads();

  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int n = 0; n < D; ++n) {
      for (int e = tid; e < r * r; e += blockDim.x) {
        T v = T(1);
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k != n) v *= Gram[k][e];
        V[e] = v;
      }
      for (int e = tid; e < m[n] * r; e += blockDim.x)
        Num[e] = mttkrp_entry<T, D>(G, m, st, Bs, r, n, e / r, e % r);
      __syncthreads();
      // New values go to Num first: every row of the old B^(n) is still read.
      for (int e = tid; e < m[n] * r; e += blockDim.x) {
        const int i = e / r, q = e % r;
        T den = T(0);
        for (int pp = 0; pp < r; ++pp) den = fma(Bs[n][i * r + pp], V[pp * r + q], den);
        const T v = Bs[n][e] * Num[e] / (den > eps ? den : eps);
        Num[e] = v > T(0) ? v : T(0);
      }
      __syncthreads();
      for (int e = tid; e < m[n] * r; e += blockDim.x) Bs[n][e] = Num[e];
      __syncthreads();
      for (int e = tid; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e % r;
        T s = T(0);
        for (int i = 0; i < m[n]; ++i) s = fma(Bs[n][i * r + a], Bs[n][i * r + b], s);
        Gram[n][e] = s;
      }
      __syncthreads();
    }
  }

  bool finite = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    T* dst = static_cast<T*>(job.B[k]);
    for (int e = tid; e < m[k] * r; e += blockDim.x) {
      dst[e] = Bs[k][e];
      finite = finite && isfinite(Bs[k][e]);
    }
  }

  if (rel_err_out != nullptr || status_out != nullptr) {
    int64_t total = 1;
#pragma unroll
    for (int k = 0; k < D; ++k) total *= m[k];
    // FP64 sums in an order that does not depend on the block size.
    __shared__ double fpart[2 * kFixedLanes];
    const double2 dg = fixed_sums2(total, [&](int64_t e) {
      int idx[D];
      int64_t rem = e;
#pragma unroll
      for (int k = D - 1; k >= 0; --k) {
        idx[k] = (int)(rem % m[k]);
        rem /= m[k];
      }
      T hat = T(0);
      for (int q = 0; q < r; ++q) {
        T prod = T(1);
#pragma unroll
        for (int k = 0; k < D; ++k) prod *= Bs[k][idx[k] * r + q];
        hat += prod;
      }
      const double g = (double)G[e];
      const double dd = g - (double)hat;
      return make_double2(dd * dd, g * g);
    }, fpart);
    if (tid == 0 && rel_err_out != nullptr)
      *rel_err_out = dg.y > 0.0 ? sqrt(dg.x / dg.y) : sqrt(dg.x);
    // The fit's status: a NaN or an overflow anywhere (in the core, or reached
    // during the sweeps) shows in the fitted factors or in the residual sums.
    if (status_out != nullptr) {
      const int ok = __syncthreads_and(finite ? 1 : 0);
      if (tid == 0)
        *status_out = (ok && isfinite(dg.x) && isfinite(dg.y)) ? NNC_OK : NNC_ERR_NONFINITE;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
nncp_kernel(const nncp_job* __restrict__ jobs, int iters, T eps, double* rel_errs,
            int* statuses) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const nncp_job job = jobs[blockIdx.x];
  int* st = statuses ? statuses + blockIdx.x : nullptr;
  // A job the host skipped (its shared memory was not sized for it).
  if (!nncp_job_valid(job)) {
    if (st != nullptr && threadIdx.x == 0) *st = NNC_ERR_INVALID_ARG;
    return;
  }
  double* out = rel_errs ? rel_errs + blockIdx.x : nullptr;
  if (job.d == 3)
    fit_one<T, 3>(job, iters, eps, smem_raw, out, st);
  else
    fit_one<T, 4>(job, iters, eps, smem_raw, out, st);
}

}  // namespace

size_t nncp_smem_bytes(const nncp_job& j, size_t elem) {
  int mmax = 0, msum = 0;
  for (int k = 0; k < j.d; ++k) {
    msum += j.m[k];
    mmax = j.m[k] > mmax ? j.m[k] : mmax;
  }
  const size_t n = (size_t)msum * j.r + (size_t)(j.d + 1) * j.r * j.r + (size_t)mmax * j.r;
  return n * elem;
}

template <typename T>
int nncp_route(int n_jobs, const nncp_job* jobs, bool skip_invalid, NncpRoute* rt) {
  *rt = NncpRoute{};
  int64_t largest = 0;
  bool l2_ok = true;  // every valid job within the two-pass kernel's limits
  size_t l2_elems = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nncp_job& j = jobs[i];
    if (!nncp_job_valid(j)) {
      if (!skip_invalid) {
        set_error_detail_text("batched nnCP: job " + std::to_string(i) +
                              " has a bad descriptor (d, m, r or a null pointer)");
        return NNC_ERR_INVALID_ARG;
      }
      ++rt->invalid;
      continue;
    }
    const size_t b = nncp_smem_bytes(j, sizeof(T));
    rt->smem = b > rt->smem ? b : rt->smem;
    int64_t e = 1;
    for (int k = 0; k < j.d; ++k) e *= j.m[k];
    largest = e > largest ? e : largest;
    if (j.d != 3 || j.r > 16) {
      l2_ok = false;
    } else {
      const size_t le = cpx_l2_elems(j);
      l2_elems = le > l2_elems ? le : l2_elems;
    }
  }
  l2_ok = l2_ok && l2_elems * sizeof(T) <= kSmemBudget;
  // The cluster form: every valid job 3-way with slabs within a CTA, and a
  // cluster per valid job on the GPU at once.
  bool cl_ok = true;
  int valid = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nncp_job& j = jobs[i];
    if (!nncp_job_valid(j)) continue;
    ++valid;
    if (j.d != 3 || cpx_cluster_elems(j) * sizeof(T) > kSmemBudget) cl_ok = false;
  }
  cl_ok = cl_ok && valid >= 1 && (int64_t)valid * cpx_cluster_ctas() <= device_sm_count();
  constexpr int64_t kTwoPassMinEntries = 16384;
  if (rt->smem > kSmemBudget) {
    if (!l2_ok) {
      set_error_detail_text("batched nnCP: a job's state exceeds one block of shared memory");
      return NNC_ERR_UNSUPPORTED;
    }
    rt->two_pass = true;
  } else {
    rt->two_pass = largest >= kTwoPassMinEntries && l2_ok;
  }
  rt->cluster = rt->two_pass && cl_ok;
  return NNC_OK;
}

template <typename T>
cudaError_t launch_nncp(const nncp_job* jobs_dev, int n_jobs, size_t smem, int iters, double eps,
                        double* rel_errs, int* statuses, cudaStream_t s, int threads) {
  if (threads < 32 || threads > kThreads || threads % 32 != 0) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit((const void*)nncp_kernel<T>, smem);
    if (e != cudaSuccess) return e;
  }
  nncp_kernel<T><<<n_jobs, threads, smem, s>>>(jobs_dev, iters, (T)eps, rel_errs, statuses);
  note_launch(s);
  return cudaGetLastError();
}

TuneKey nncp_tune_key(const nncp_job* jobs, int n_jobs, size_t elem) {
  long long work = 1;
  for (int i = 0; i < n_jobs; ++i) {
    if (!nncp_job_valid(jobs[i])) continue;
    long long w = jobs[i].r;  // one sweep: every entry of the core once per mode and q
    for (int k = 0; k < jobs[i].d; ++k) w *= jobs[i].m[k];
    work = w > work ? w : work;
  }
  return TuneKey{kTuneNncp, (int)elem, size_class(work), size_class(n_jobs)};
}

template cudaError_t launch_nncp<float>(const nncp_job*, int, size_t, int, double, double*,
                                        int*, cudaStream_t, int);
template cudaError_t launch_nncp<double>(const nncp_job*, int, size_t, int, double, double*,
                                         int*, cudaStream_t, int);
template int nncp_route<float>(int, const nncp_job*, bool, NncpRoute*);
template int nncp_route<double>(int, const nncp_job*, bool, NncpRoute*);

}  // namespace nnc
