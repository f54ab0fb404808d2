// Differentiation form: the adjoint of the lifted loss and a block
// projected-gradient fit of it.
//
// The objective of Eq. nnCANDELINC with the CPD of the core substituted,
//   L = 1/2 ||X - I x_n A^(n)||^2,  A^(n) = F^(n) B^(n)  (d = 3 or 4),
// has, with V_n = Hadamard_{k!=n} A^(k)T A^(k) and
//   MT_n = unfold_n(X) KR_{k!=n}(A^(k)) = unfold_n(Z_n) KR_{k!=n}(B^(k)),
//   Z_n  = X x_{k!=n} F^(k)T        (the Tucker-compressed tensor),
// the gradients dL/dA^(n) = A^(n) V_n - MT_n, dL/dF^(n) = (dL/dA^(n)) B^(n)T
// and dL/dB^(n) = F^(n)T dL/dA^(n). The KR identity holds because
// KR_k(F^(k) B^(k)) = (kron_k F^(k)) KR_k(B^(k)).
//
// X is read twice per gradient: T_last = X x_d F^(d)T serves every Z_n with
// n < d (further mode products on the compressed tensor), and
// T_first = X x_1 F^(1)T serves Z_d. FP32 runs both passes on the TF32x3
// tensor-core kernel with X viewed as 3-way (N_1, N_2 ... N_{d-1}, N_d); FP64
// and FP32_SIMT run the SIMT mode products. The loss comes out of the same
// terms in FP64: L = 1/2 ||X||^2 - <MT_n, A^(n)> + 1/2 sum(V_n .* A^(n)T A^(n)).
//
// The fit (block-coordinate projected gradient, the builder's reading since
// the paper gives no first-order method): for n = 1..d, with MT_n and V_n,
//   F^(n) <- max(F^(n) - (A V - MT) B^(n)T / L_F, 0),  L_F = lmax(B V B^T),
//   B^(n) <- max(B^(n) - F^(n)T (A V - MT) / L_B, 0),  L_B = lmax(F^T F) lmax(V),
// with lmax from 30 FP64 power iterations (all-ones start, Rayleigh quotient).
// MT_n does not involve mode n, so one Z_n serves both blocks of mode n; the
// Gauss-Seidel order still needs only two passes over X per step (T_last before
// mode 1, T_first after mode d-1).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "lifted.cuh"
#include "residual.cuh"
#include "sweep.cuh"
#include "tc_ttm.cuh"

namespace nnc {
namespace {

constexpr int kMaxD = 4;
constexpr int kPowerIters = 30;

inline unsigned grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

// ---- small dense kernels ------------------------------------------------------

// C[i, j] = sum_k A[i as_i + k as_k] B[k bs_k + j bs_j] - (D ? D[i, j] : 0)
// for i < M, j < N (C and D row-major, ld N). One thread per output.
template <typename T>
__global__ void small_gemm_kernel(int M, int N, int K, const T* __restrict__ A, int64_t as_i,
                                  int64_t as_k, const T* __restrict__ B, int64_t bs_k,
                                  int64_t bs_j, const T* __restrict__ D, T* __restrict__ C) {
  const int64_t n = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e % N;
    T acc = T(0);
    for (int k = 0; k < K; ++k) acc = fma(A[i * as_i + k * as_k], B[k * bs_k + j * bs_j], acc);
    C[e] = D ? acc - D[e] : acc;
  }
}

template <typename T>
cudaError_t small_gemm(int M, int N, int K, const T* A, int64_t as_i, int64_t as_k, const T* B,
                       int64_t bs_k, int64_t bs_j, const T* D, T* C, cudaStream_t s) {
  small_gemm_kernel<T><<<grid_for((int64_t)M * N, 256), 256, 0, s>>>(M, N, K, A, as_i, as_k, B,
                                                                      bs_k, bs_j, D, C);
  note_launch(s);
  return cudaGetLastError();
}

// out[t, q] = prod_k B_k[idx_k(t), q], t in C order over the listed modes (the
// last one fastest); a single row of ones when no mode is listed.
template <typename T>
struct KrArgs {
  const T* B[kMaxD];
  int m[kMaxD];
  int nk;
  int r;
  int64_t rows;
  T* out;
};

template <typename T>
__global__ void kr_kernel(KrArgs<T> a) {
  const int64_t n = a.rows * a.r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % a.r);
    int64_t t = e / a.r;
    T v = T(1);
    for (int k = a.nk - 1; k >= 0; --k) {
      const int ik = (int)(t % a.m[k]);
      t /= a.m[k];
      v *= a.B[k][(int64_t)ik * a.r + q];
    }
    a.out[e] = v;
  }
}

// MT[i, q] = sum_p W[(p N + i) r + q] Kpre[p r + q], p in order.
template <typename T>
__global__ void weighted_sum_p_kernel(const T* __restrict__ W, const T* __restrict__ Kpre,
                                      int64_t P, int64_t N, int r, T* __restrict__ MT) {
  const int64_t n = N * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % r);
    T acc = T(0);
    for (int64_t p = 0; p < P; ++p) acc = fma(W[p * n + e], Kpre[p * r + q], acc);
    MT[e] = acc;
  }
}

// out (C x R) = in^T, in R x C row-major.
template <typename T>
__global__ void transpose_small_kernel(const T* __restrict__ in, int R, int64_t C,
                                       T* __restrict__ out) {
  const int64_t n = (int64_t)R * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / R, rr = e % R;
    out[e] = in[rr * C + c];
  }
}

// I (r x r).
template <typename T>
__global__ void identity_kernel(T* I, int r) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) I[e] = (e / r == e % r) ? T(1) : T(0);
}

// out = ||R|| / a (||R|| when a is null), n entries, FP64 sum in a fixed
// order; also trace[*counter] (then *counter + 1) when a trace is given.
template <typename T>
__global__ void rel_norm_kernel(const T* __restrict__ R, int64_t n, const double* __restrict__ a,
                                double* out, double* trace, int* counter) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += (double)R[e] * (double)R[e];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double v = a ? sqrt(s) / a[0] : sqrt(s);
    out[0] = v;
    if (counter) trace_record(counter, trace, 1, v, true);
  }
}

// V = Hadamard product of the listed r x r matrices (all ones if none).
template <typename T>
struct HadArgs {
  const T* M[kMaxD];
  int nk;
  int r;
  T* out;
};

template <typename T>
__global__ void hadamard_kernel(HadArgs<T> a) {
  for (int e = threadIdx.x; e < a.r * a.r; e += blockDim.x) {
    T v = T(1);
    for (int k = 0; k < a.nk; ++k) v *= a.M[k][e];
    a.out[e] = v;
  }
}

// out_b = lmax(H_b) for the matrix b = blockIdx.x of the launch (H_0: n0 x n0,
// H_1: n1 x n1, n <= 64): kPowerIters FP64 power iterations from the
// normalised all-ones vector, then the Rayleigh quotient; 0 if an iterate maps
// to zero. One warp per matrix: lane l owns rows l and l + 32 of H (kept in
// shared memory with an odd row stride) and the same entries of v, which the
// products fetch by shuffles. FP64 is slow on this GPU, and an iteration then
// needs no block barrier: one shuffle sum for the norm and one reciprocal.
template <typename T>
__global__ void __launch_bounds__(32) power_iter_kernel(const T* __restrict__ H0, int n0,
                                                         double* out0, const T* __restrict__ H1,
                                                         int n1, double* out1) {
  __shared__ double h[64 * 65];
  const T* H = blockIdx.x == 0 ? H0 : H1;
  const int n = blockIdx.x == 0 ? n0 : n1;
  double* out = blockIdx.x == 0 ? out0 : out1;
  const int lane = threadIdx.x, ld = n + 1;
  for (int e = lane; e < n * n; e += 32) h[(e / n) * ld + e % n] = (double)H[e];
  __syncwarp();
  const int r0 = lane, r1 = lane + 32;
  const bool has0 = r0 < n, has1 = r1 < n;
  const double v0i = 1.0 / sqrt((double)n);
  double v0 = has0 ? v0i : 0.0, v1 = has1 ? v0i : 0.0;  // v[r0], v[r1]
  double w0 = 0.0, w1 = 0.0;
  auto matvec = [&]() {  // (w0, w1) = rows r0, r1 of H v
    double a0 = 0.0, b0 = 0.0, a1 = 0.0, b1 = 0.0;
    int j = 0;
    for (; j + 1 < n; j += 2) {
      const double x = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
      const double y = __shfl_sync(0xffffffffu, j + 1 < 32 ? v0 : v1, (j + 1) & 31);
      if (has0) {
        a0 = fma(h[r0 * ld + j], x, a0);
        b0 = fma(h[r0 * ld + j + 1], y, b0);
      }
      if (has1) {
        a1 = fma(h[r1 * ld + j], x, a1);
        b1 = fma(h[r1 * ld + j + 1], y, b1);
      }
    }
    if (j < n) {
      const double x = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
      if (has0) a0 = fma(h[r0 * ld + j], x, a0);
      if (has1) a1 = fma(h[r1 * ld + j], x, a1);
    }
    w0 = a0 + b0;
    w1 = a1 + b1;
  };
  for (int it = 0; it < kPowerIters; ++it) {
    matvec();
    const double nrm = sqrt(warp_sum(w0 * w0 + w1 * w1));
    if (!(nrm > 0.0)) {
      if (lane == 0) out[0] = 0.0;
      return;
    }
    const double inv = 1.0 / nrm;
    v0 = w0 * inv;
    v1 = w1 * inv;
  }
  matvec();
  const double q = warp_sum(v0 * w0 + v1 * w1);
  if (lane == 0) out[0] = q;
}

// P <- max(P - G / L, 0) when L > 0, with L = L1[0] (times L2[0] if given).
template <typename T>
__global__ void pg_update_kernel(T* __restrict__ P, const T* __restrict__ G, int64_t n,
                                 const double* __restrict__ L1, const double* __restrict__ L2) {
  const double l = L2 ? L1[0] * L2[0] : L1[0];
  if (!(l > 0.0)) return;
  const T inv = (T)(1.0 / l);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = P[e] - G[e] * inv;
    P[e] = v > T(0) ? v : T(0);
  }
}

// *out = 1/2 x2 - <MT, A> + 1/2 sum(V .* AtA), FP64 sums in a fixed order (one
// block); also trace[*counter] (then *counter + 1) when a trace is given.
template <typename T>
__global__ void lifted_loss_kernel(const T* __restrict__ MT, const T* __restrict__ A, int64_t n,
                                   const T* __restrict__ V, const T* __restrict__ AtA, int rr,
                                   const double* __restrict__ x2, double* out, double* trace,
                                   int* counter, int rel) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) a += (double)MT[e] * (double)A[e];
  for (int e = threadIdx.x; e < rr; e += blockDim.x) b += (double)V[e] * (double)AtA[e];
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    double v = 0.5 * x2[0] - a + 0.5 * b;
    const bool finite = isfinite(v);
    if (rel) v = sqrt((v > 0.0 ? 2.0 * v : 0.0) / x2[0]);  // ||X - X_hat|| / ||X||
    out[0] = v;
    if (counter) trace_record(counter, trace, 1, v, finite);
  }
}

// ---- the workspace -------------------------------------------------------------

// A side stream and a fork/join pair of events for the branches captured in a
// replayed sweep (each record of an event marks the point the next wait joins).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t m_ready = nullptr, g_ready = nullptr;  // the pending core update's steps
  int init() {
    NNC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&m_ready, cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g_ready, cudaEventDisableTiming));
    return NNC_OK;
  }
  ~SideStream() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (m_ready) cudaEventDestroy(m_ready);
    if (g_ready) cudaEventDestroy(g_ready);
    if (s) cudaStreamDestroy(s);
  }
};

template <typename T>
struct Work {
  int d = 0, r = 0;
  int64_t N[kMaxD] = {};
  int m[kMaxD] = {};
  const T* X = nullptr;
  bool tc = false;
  tc::TcPlan plan;
  T *Tlast = nullptr, *Tfirst = nullptr, *U0 = nullptr, *Z0 = nullptr, *Z1 = nullptr;
  T* W = nullptr;
  T *Kpre = nullptr, *Kpost = nullptr, *MT = nullptr, *gA = nullptr, *tmp = nullptr;
  T *V = nullptr, *H = nullptr, *S = nullptr;
  T* tmp2 = nullptr;  // B V of a projected-gradient block, beside the gradient chain in tmp
  T* split = nullptr;  // partial sums of mode products whose grid would not fill the GPU
  size_t split_cap = 0;
  T* A[kMaxD] = {};
  T* AtA[kMaxD] = {};
  double *stats_part = nullptr, *stats = nullptr, *Ls = nullptr;
};

int64_t prod(const int64_t* v, int a, int b) {  // v[a] ... v[b-1]
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= v[i];
  return p;
}

template <typename T>
int setup(Work<T>& w, const T* X, int d, const int64_t* dims, const int* m, int r, bool want_tc,
          Scratch& sc, cudaStream_t s) {
  w.d = d;
  w.r = r;
  w.X = X;
  int64_t nmax = 0;
  int mmax = 0;
  for (int k = 0; k < d; ++k) {
    w.N[k] = dims[k];
    w.m[k] = m[k];
    nmax = dims[k] > nmax ? dims[k] : nmax;
    mmax = m[k] > mmax ? m[k] : mmax;
  }
  const int64_t nX = prod(dims, 0, d);
  const int64_t tl = nX / dims[d - 1] * m[d - 1];
  const int64_t tf = nX / dims[0] * m[0];
  // Largest intermediate of the Z chains: the first product of each chain.
  int64_t zmax = 1;
  for (int n = 0; n < d; ++n) {
    int64_t cur[kMaxD];
    for (int k = 0; k < d; ++k) cur[k] = dims[k];
    if (n < d - 1) cur[d - 1] = m[d - 1];
    else cur[0] = m[0];
    for (int k = 0; k < d; ++k) {
      if (k == n || (n < d - 1 && k == d - 1) || (n == d - 1 && k == 0)) continue;
      cur[k] = m[k];
      const int64_t sz = prod(cur, 0, d);
      zmax = sz > zmax ? sz : zmax;
    }
  }
  int64_t pmax = 1;  // largest product of other modes' ranks
  for (int n = 0; n < d; ++n) {
    int64_t p = 1;
    for (int k = 0; k < d; ++k)
      if (k != n) p *= m[k];
    pmax = p > pmax ? p : pmax;
  }
  NNC_TRY(sc.get(&w.Tlast, (size_t)tl));
  NNC_TRY(sc.get(&w.Tfirst, (size_t)tf));
  NNC_TRY(sc.get(&w.U0, (size_t)(tl / dims[0] * m[0])));
  NNC_TRY(sc.get(&w.Z0, (size_t)zmax));
  NNC_TRY(sc.get(&w.Z1, (size_t)zmax));
  NNC_TRY(sc.get(&w.W, (size_t)(pmax * nmax * r)));
  NNC_TRY(sc.get(&w.Kpre, (size_t)(pmax * r)));
  NNC_TRY(sc.get(&w.Kpost, (size_t)(pmax * r)));
  NNC_TRY(sc.get(&w.MT, (size_t)(nmax * r)));
  NNC_TRY(sc.get(&w.gA, (size_t)(nmax * r)));
  NNC_TRY(sc.get(&w.tmp, (size_t)(nmax * (mmax > r ? mmax : r))));
  NNC_TRY(sc.get(&w.tmp2, (size_t)mmax * r));
  NNC_TRY(sc.get(&w.V, (size_t)(r * r)));
  NNC_TRY(sc.get(&w.H, (size_t)(mmax * mmax > r * r ? mmax * mmax : r * r)));
  NNC_TRY(sc.get(&w.S, (size_t)(mmax * mmax)));
  w.split_cap = (size_t)1 << 22;
  NNC_TRY(sc.get(&w.split, w.split_cap));
  for (int k = 0; k < d; ++k) {
    NNC_TRY(sc.get(&w.A[k], (size_t)(dims[k] * r)));
    NNC_TRY(sc.get(&w.AtA[k], (size_t)(r * r)));
  }
  NNC_TRY(sc.get(&w.stats_part, 3 * kStatBlocks));
  NNC_TRY(sc.get(&w.stats, 3));
  NNC_TRY(sc.get(&w.Ls, 4));
  NNC_CUDA_TRY(launch_tensor_stats<T>(X, nX, w.stats_part, w.stats, s));
  double st[3];
  NNC_CUDA_TRY(cudaMemcpyAsync(st, w.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (st[2] > 0.0) return NNC_ERR_NONFINITE;
  w.tc = false;
  if constexpr (std::is_same<T, float>::value) {
    if (want_tc) {
      const int st2 = w.plan.init(tc::kKindTf32x3, X, dims[0], prod(dims, 1, d - 1),
                                  dims[d - 1], m[0], m[d - 1], sc, s);
      if (st2 == NNC_OK) w.tc = true;
      else if (st2 != NNC_ERR_UNSUPPORTED) return st2;
    }
  }
  return NNC_OK;
}

// T_last = X x_d F^(d)T laid out (N_1, ..., N_{d-1}, m_d).
template <typename T>
int pass_last(Work<T>& w, const T* Fd, cudaStream_t s) {
  const int d = w.d;
  if constexpr (std::is_same<T, float>::value) {
    if (w.tc) return w.plan.pass3(Fd, w.Tlast, s, /*convert=*/true);
  }
  NNC_CUDA_TRY(launch_ttm<T>(w.X, prod(w.N, 0, d - 1), (int)w.N[d - 1], 1, Fd, w.m[d - 1], 1,
                             w.m[d - 1], w.Tlast, nullptr, 0, s));
  return NNC_OK;
}

// T_first = X x_1 F^(1)T laid out (m_1, N_2, ..., N_d).
template <typename T>
int pass_first(Work<T>& w, const T* F1, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (w.tc) return w.plan.pass1(F1, w.Tfirst, s, /*convert=*/true);
  }
  NNC_CUDA_TRY(launch_ttm<T>(w.X, 1, (int)w.N[0], prod(w.N, 1, w.d), F1, w.m[0], 1, w.m[0],
                             w.Tfirst, nullptr, 0, s));
  return NNC_OK;
}

// U0 = T_last x_1 F^(1)T, laid out (m_1, N_2, ..., N_{d-1}, m_d): shared by every
// Z_n with 1 < n < d (its F^(1) is final for the step once mode 1 is done).
template <typename T>
int make_u0(Work<T>& w, const T* F1, cudaStream_t s) {
  const int d = w.d;
  auto ttm = w.tc ? launch_ttm_tc<T> : launch_ttm<T>;
  NNC_CUDA_TRY(ttm(w.Tlast, 1, (int)w.N[0], prod(w.N, 1, d - 1) * w.m[d - 1], F1, w.m[0], 1,
                   w.m[0], w.U0, w.split, w.split_cap, s));
  return NNC_OK;
}

// Z_n by mode products with the current factors, laid out (m_1 .. N_n .. m_d):
// from T_last (n = 1), U0 (1 < n < d) or T_first (n = d).
template <typename T>
int z_chain(Work<T>& w, int n, T* const* F, const T** zout, cudaStream_t s) {
  const int d = w.d;
  int64_t cur[kMaxD];
  for (int k = 0; k < d; ++k) cur[k] = w.N[k];
  const T* src;
  int first = 0;  // modes [first, last) other than n are contracted here
  int last = d;
  if (n == d - 1) {
    cur[0] = w.m[0];
    src = w.Tfirst;
    first = 1;
  } else if (n == 0) {
    cur[d - 1] = w.m[d - 1];
    src = w.Tlast;
    last = d - 1;
  } else {
    cur[0] = w.m[0];
    cur[d - 1] = w.m[d - 1];
    src = w.U0;
    first = 1;
    last = d - 1;
  }
  T* bufs[2] = {w.Z0, w.Z1};
  int b = 0;
  auto ttm = w.tc ? launch_ttm_tc<T> : launch_ttm<T>;
  for (int k = first; k < last; ++k) {
    if (k == n) continue;
    NNC_CUDA_TRY(ttm(src, prod(cur, 0, k), (int)cur[k], prod(cur, k + 1, d), F[k], w.m[k], 1,
                     w.m[k], bufs[b], w.split, w.split_cap, s));
    cur[k] = w.m[k];
    src = bufs[b];
    b ^= 1;
  }
  *zout = src;
  return NNC_OK;
}

// MT_n = unfold_n(Z_n) KR_{k!=n}(B^(k)) into w.MT; V_n into w.V.
template <typename T>
int mttkrp_and_v(Work<T>& w, int n, const T* Z, T* const* B, cudaStream_t s) {
  const int d = w.d, r = w.r;
  KrArgs<T> pre{}, post{};
  pre.r = post.r = r;
  pre.out = w.Kpre;
  post.out = w.Kpost;
  pre.rows = post.rows = 1;
  for (int k = 0; k < d; ++k) {
    if (k < n) {
      pre.B[pre.nk] = B[k];
      pre.m[pre.nk++] = w.m[k];
      pre.rows *= w.m[k];
    } else if (k > n) {
      post.B[post.nk] = B[k];
      post.m[post.nk++] = w.m[k];
      post.rows *= w.m[k];
    }
  }
  kr_kernel<T><<<grid_for(pre.rows * r, 256), 256, 0, s>>>(pre);
  note_launch(s);
  kr_kernel<T><<<grid_for(post.rows * r, 256), 256, 0, s>>>(post);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  if (post.rows == 1) {
    // Last mode: MT^T (r x N) = Kpre^T unfold(Z), one mode product over p;
    // then MT = (MT^T)^T.
    NNC_CUDA_TRY(launch_ttm<T>(Z, 1, (int)pre.rows, w.N[n], w.Kpre, r, 1, r, w.W, w.split,
                               w.split_cap, s));
    transpose_small_kernel<T><<<grid_for(w.N[n] * r, 256), 256, 0, s>>>(w.W, r, w.N[n], w.MT);
    note_launch(s);
  } else {
    // W[p, i, q] = sum_s Z[p, i, s] Kpost[s, q];  MT[i, q] = sum_p W[p, i, q] Kpre[p, q]
    T* Wout = pre.rows == 1 ? w.MT : w.W;
    NNC_CUDA_TRY(launch_ttm<T>(Z, pre.rows * w.N[n], (int)post.rows, 1, w.Kpost, r, 1, r, Wout,
                               w.split, w.split_cap, s));
    if (pre.rows > 1) {
      weighted_sum_p_kernel<T><<<grid_for(w.N[n] * r, 256), 256, 0, s>>>(w.W, w.Kpre, pre.rows,
                                                                           w.N[n], r, w.MT);
      note_launch(s);
    }
  }
  HadArgs<T> h{};
  h.r = r;
  h.out = w.V;
  for (int k = 0; k < d; ++k)
    if (k != n) h.M[h.nk++] = w.AtA[k];
  hadamard_kernel<T><<<1, 256, 0, s>>>(h);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

// A^(k) = F^(k) B^(k) and A^(k)T A^(k).
template <typename T>
int refresh_a(Work<T>& w, int k, const T* Fk, const T* Bk, cudaStream_t s) {
  NNC_CUDA_TRY(launch_lift<T>(Fk, Bk, w.N[k], w.m[k], w.r, w.A[k], s));
  NNC_TRY(launch_gram<T>(w.A[k], w.N[k], w.r, w.AtA[k], s));
  return NNC_OK;
}

// gA = A^(n) V - MT (N_n x r) into w.gA.
template <typename T>
int grad_a(Work<T>& w, int n, cudaStream_t s) {
  const int r = w.r;
  NNC_CUDA_TRY(small_gemm<T>((int)w.N[n], r, r, w.A[n], r, 1, w.V, r, 1, w.MT, w.gA, s));
  return NNC_OK;
}

// One block pair (F^(n), then B^(n)) of the projected-gradient step. The step
// sizes (power iterations on small FP64 chains) need nothing from the
// gradient chain, so with a side stream each runs beside it and is joined
// before the update that uses it (the same launches either way).
template <typename T>
int pg_mode(Work<T>& w, int n, T* const* F, T* const* B, cudaStream_t s, SideStream* side) {
  const int r = w.r, mn = w.m[n];
  const int64_t Nn = w.N[n];
  const cudaStream_t ls = side ? side->s : s;
  auto fork = [&]() -> int {
    if (!side) return NNC_OK;
    NNC_CUDA_TRY(cudaEventRecord(side->fork, s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
    return NNC_OK;
  };
  auto join = [&]() -> int {
    if (!side) return NNC_OK;
    NNC_CUDA_TRY(cudaEventRecord(side->join, side->s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(s, side->join, 0));
    return NNC_OK;
  };
  // L_F = lmax(B V B^T) and lmax(V) (one launch): tmp2 = B V (m x r), H = tmp2 B^T (m x m)
  NNC_TRY(fork());
  NNC_CUDA_TRY(small_gemm<T>(mn, r, r, B[n], r, 1, w.V, r, 1, nullptr, w.tmp2, ls));
  NNC_CUDA_TRY(small_gemm<T>(mn, mn, r, w.tmp2, r, 1, B[n], 1, r, nullptr, w.H, ls));
  power_iter_kernel<T><<<2, 32, 0, ls>>>(w.H, mn, w.Ls + 0, w.V, r, w.Ls + 1);
  note_launch(ls);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_TRY(grad_a(w, n, s));
  // gF = gA B^T (N x m) into tmp
  NNC_CUDA_TRY(small_gemm<T>((int)Nn, mn, r, w.gA, r, 1, B[n], 1, r, nullptr, w.tmp, s));
  NNC_TRY(join());
  pg_update_kernel<T><<<grid_for(Nn * mn, 256), 256, 0, s>>>(F[n], w.tmp, Nn * mn, w.Ls + 0,
                                                               nullptr);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_CUDA_TRY(launch_lift<T>(F[n], B[n], Nn, mn, r, w.A[n], s));
  // L_B = lmax(F^T F) lmax(V)
  NNC_TRY(fork());
  NNC_TRY(launch_gram<T>(F[n], Nn, mn, w.S, ls));
  power_iter_kernel<T><<<1, 32, 0, ls>>>(w.S, mn, w.Ls + 2, w.S, mn, w.Ls + 2);
  note_launch(ls);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_TRY(grad_a(w, n, s));
  // gB = F^T gA (m x r) into tmp
  NNC_CUDA_TRY(small_gemm<T>(mn, r, (int)Nn, F[n], 1, mn, w.gA, r, 1, nullptr, w.tmp, s));
  NNC_TRY(join());
  pg_update_kernel<T><<<grid_for((int64_t)mn * r, 256), 256, 0, s>>>(B[n], w.tmp, (int64_t)mn * r,
                                                                      w.Ls + 2, w.Ls + 1);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_TRY(refresh_a(w, n, F[n], B[n], s));
  return NNC_OK;
}

template <typename T>
int loss_into(Work<T>& w, int n, double* out, double* trace, int* counter, cudaStream_t s,
              int rel = 0) {
  lifted_loss_kernel<T><<<1, 256, 0, s>>>(w.MT, w.A[n], w.N[n] * w.r, w.V, w.AtA[n], w.r * w.r,
                                          w.stats, out, trace, counter, rel);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int check_tc(Work<T>& w, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (w.tc) return w.plan.check(s);
  }
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  return NNC_OK;
}

}  // namespace

template <typename T>
int lifted_grad(const T* X, int d, const int64_t* dims, const int* m, int r, bool tensor_cores,
                T* const* F, T* const* B, T* const* gF, T* const* gB, double* loss,
                cudaStream_t s) {
  Scratch sc(s);
  Work<T> w;
  NNC_TRY(setup(w, X, d, dims, m, r, tensor_cores, sc, s));
  for (int k = 0; k < d; ++k) NNC_TRY(refresh_a(w, k, F[k], B[k], s));
  const bool grads = gF != nullptr;
  double* dloss = w.Ls + 3;
  NNC_TRY(pass_last(w, F[d - 1], s));
  if (grads) {
    NNC_TRY(pass_first(w, F[0], s));
    NNC_TRY(make_u0(w, F[0], s));
  }
  for (int n = 0; n < (grads ? d : 1); ++n) {
    const T* Z = nullptr;
    NNC_TRY(z_chain(w, n, F, &Z, s));
    NNC_TRY(mttkrp_and_v(w, n, Z, B, s));
    if (n == 0) NNC_TRY(loss_into(w, 0, dloss, nullptr, nullptr, s));
    if (!grads) break;
    NNC_TRY(grad_a(w, n, s));
    const int mn = m[n];
    NNC_CUDA_TRY(small_gemm<T>((int)dims[n], mn, r, w.gA, r, 1, B[n], 1, r, nullptr, gF[n], s));
    NNC_CUDA_TRY(small_gemm<T>(mn, r, (int)dims[n], F[n], 1, mn, w.gA, r, 1, nullptr, gB[n], s));
  }
  NNC_TRY(check_tc(w, s));
  if (loss) {
    NNC_CUDA_TRY(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
    NNC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return NNC_OK;
}

namespace {

// One projected-gradient step (two passes over X), stream-ordered on s.
template <typename T>
int pg_step(Work<T>& w, T* const* F, T* const* B, double* last, double* trace, int* counter,
            cudaStream_t s, SideStream* side) {
  const int d = w.d;
  NNC_TRY(pass_last(w, F[d - 1], s));
  for (int n = 0; n < d; ++n) {
    if (n == d - 1) NNC_TRY(pass_first(w, F[0], s));
    const T* Z = nullptr;
    NNC_TRY(z_chain(w, n, F, &Z, s));
    NNC_TRY(mttkrp_and_v(w, n, Z, B, s));
    NNC_TRY(pg_mode(w, n, F, B, s, side));
    if (n == 0 && d > 2) NNC_TRY(make_u0(w, F[0], s));
  }
  // MT_d and V_d do not involve mode d: the loss at the new point.
  return loss_into(w, d - 1, last, trace, counter, s);
}

// Private stream, graph and events of the replay loop.
struct PgGraph {
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ~PgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (cs) cudaStreamDestroy(cs);
  }
};

}  // namespace

template <typename T>
int lifted_pg_fit(const T* X, int d, const int64_t* dims, const int* m, int r, bool tensor_cores,
                  int steps, T* const* F, T* const* B, double* trace, double* loss,
                  cudaStream_t s) {
  Scratch sc(s);
  Work<T> w;
  NNC_TRY(setup(w, X, d, dims, m, r, tensor_cores, sc, s));
  for (int k = 0; k < d; ++k) NNC_TRY(refresh_a(w, k, F[k], B[k], s));
  double* last = w.Ls + 3;
  int* counter = nullptr;
  NNC_TRY(sc.get(&counter, 2));
  NNC_CUDA_TRY(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  if (steps > 0) {
    // One step is captured as a CUDA graph on a private stream and replayed;
    // the trace slot advances through the device counter.
    PgGraph g;
    SideStream side;
    NNC_TRY(side.init());
    NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventRecord(g.fork, s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(g.cs, g.fork, 0));
    NNC_CUDA_TRY(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
    const int cap = pg_step(w, F, B, last, trace, counter, g.cs, &side);
    const cudaError_t end_e = cudaStreamEndCapture(g.cs, &g.graph);
    if (cap != NNC_OK) return cap;
    NNC_CUDA_TRY(end_e);
    NNC_CUDA_TRY(cudaGraphInstantiate(&g.exec, g.graph, 0));
    size_t nn = 0;
    NNC_CUDA_TRY(cudaGraphGetNodes(g.graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    NNC_CUDA_TRY(cudaGraphGetNodes(g.graph, nodes.data(), &nn));
    long long kernels = 0;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      NNC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
      if (ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    for (int t = 0; t < steps; ++t) NNC_CUDA_TRY(cudaGraphLaunch(g.exec, g.cs));
    note_graph_launches(kernels * steps);
    NNC_CUDA_TRY(cudaEventRecord(g.join, g.cs));
    NNC_CUDA_TRY(cudaStreamWaitEvent(s, g.join, 0));
    NNC_CUDA_TRY(cudaStreamSynchronize(g.cs));
  }
  NNC_TRY(check_tc(w, s));
  NNC_TRY(check_trace_finite(counter, s, "candelinc_pg_fit"));
  if (loss) {
    if (steps == 0) {
      *loss = NAN;
    } else {
      NNC_CUDA_TRY(cudaMemcpyAsync(loss, last, sizeof(double), cudaMemcpyDeviceToHost, s));
      NNC_CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  return NNC_OK;
}

namespace {

// Captures `body` (stream-ordered work on a private stream) once as a CUDA
// graph and replays it `count` times after the work queued on s; `after(t,
// cs)`, if given, queues work on the private stream after replay t.
struct NoAfter {
  int operator()(int, cudaStream_t) const { return NNC_OK; }
};
template <typename Body, typename After = NoAfter>
int replay(int count, cudaStream_t s, Body body, After after = After()) {
  if (count <= 0) return NNC_OK;
  PgGraph g;
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventRecord(g.fork, s));
  NNC_CUDA_TRY(cudaStreamWaitEvent(g.cs, g.fork, 0));
  NNC_CUDA_TRY(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
  const int cap = body(g.cs);
  const cudaError_t end_e = cudaStreamEndCapture(g.cs, &g.graph);
  if (cap != NNC_OK) return cap;
  NNC_CUDA_TRY(end_e);
  NNC_CUDA_TRY(cudaGraphInstantiate(&g.exec, g.graph, 0));
  size_t nn = 0;
  NNC_CUDA_TRY(cudaGraphGetNodes(g.graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  NNC_CUDA_TRY(cudaGraphGetNodes(g.graph, nodes.data(), &nn));
  long long kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    NNC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  for (int t = 0; t < count; ++t) {
    NNC_CUDA_TRY(cudaGraphLaunch(g.exec, g.cs));
    NNC_TRY(after(t, g.cs));
  }
  note_graph_launches(kernels * count);
  NNC_CUDA_TRY(cudaEventRecord(g.join, g.cs));
  NNC_CUDA_TRY(cudaStreamWaitEvent(s, g.join, 0));
  NNC_CUDA_TRY(cudaStreamSynchronize(g.cs));
  return NNC_OK;
}

// Kernel nodes of a captured graph.
int graph_kernels(cudaGraph_t graph, long long* kernels) {
  size_t nn = 0;
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nn));
  *kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    NNC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++*kernels;
  }
  return NNC_OK;
}

// Captures `first`, `rest` and `last` (stream-ordered work on one private
// stream) as three CUDA graphs and runs first once, rest count - 1 times and
// last once, after the work queued on s (count >= 1).
template <typename First, typename Rest, typename Last>
int replay_pipelined(int count, cudaStream_t s, First first, Rest rest, Last last) {
  if (count <= 0) return NNC_OK;
  PgGraph g[3];
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g[0].cs, cudaStreamNonBlocking));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g[0].fork, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g[0].join, cudaEventDisableTiming));
  cudaStream_t cs = g[0].cs;
  NNC_CUDA_TRY(cudaEventRecord(g[0].fork, s));
  NNC_CUDA_TRY(cudaStreamWaitEvent(cs, g[0].fork, 0));
  long long kernels[3] = {0, 0, 0};
  auto capture = [&](int i, auto& body) -> int {
    NNC_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int st = body(cs);
    const cudaError_t e = cudaStreamEndCapture(cs, &g[i].graph);
    if (st != NNC_OK) return st;
    NNC_CUDA_TRY(e);
    NNC_CUDA_TRY(cudaGraphInstantiate(&g[i].exec, g[i].graph, 0));
    return graph_kernels(g[i].graph, &kernels[i]);
  };
  NNC_TRY(capture(0, first));
  NNC_TRY(capture(1, rest));
  NNC_TRY(capture(2, last));
  NNC_CUDA_TRY(cudaGraphLaunch(g[0].exec, cs));
  for (int t = 1; t < count; ++t) NNC_CUDA_TRY(cudaGraphLaunch(g[1].exec, cs));
  NNC_CUDA_TRY(cudaGraphLaunch(g[2].exec, cs));
  note_graph_launches(kernels[0] + kernels[1] * (count - 1) + kernels[2]);
  NNC_CUDA_TRY(cudaEventRecord(g[0].join, cs));
  NNC_CUDA_TRY(cudaStreamWaitEvent(s, g[0].join, 0));
  NNC_CUDA_TRY(cudaStreamSynchronize(cs));
  return NNC_OK;
}

}  // namespace

// nnCPD of X itself (Alg. 2, first step): the MU sweep of the core nnCPD with
// X in place of G, A^(n) <- max(A^(n) .* MT_n / max(A^(n) V_n, eps), 0) for
// n = 1..d. MT_n comes from the lifted machinery with F := A and B := I_r
// (so m := r): two passes over X per sweep, T_last = X x_d A^(d)T serving
// modes 1..d-1 and T_first = X x_1 A^(1)T mode d. trace[t] (device, optional)
// = ||X - I x_k A^(k)|| / ||X|| after sweep t by the identity in FP64.
template <typename T>
int nncp_tensor_fit(const T* X, int d, const int64_t* dims, int r, bool tensor_cores, int iters,
                    double eps, int exact_every, T* const* A, double* trace, double* rel_err,
                    cudaStream_t s) {
  Scratch sc(s);
  Work<T> w;
  int m[kMaxD];
  for (int k = 0; k < d; ++k) m[k] = r;
  NNC_TRY(setup(w, X, d, dims, m, r, tensor_cores, sc, s));
  T* I = nullptr;
  NNC_TRY(sc.get(&I, (size_t)r * r));
  identity_kernel<T><<<1, 256, 0, s>>>(I, r);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  T* B[kMaxD];
  for (int k = 0; k < d; ++k) B[k] = I;
  for (int k = 0; k < d; ++k) NNC_TRY(refresh_a(w, k, A[k], B[k], s));
  int* counter = nullptr;
  NNC_TRY(sc.get(&counter, 2));
  NNC_CUDA_TRY(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  double* last = w.Ls + 3;
  // Exact checkpoints (nnc_opts exact_every): after every exact_every-th sweep
  // and the last, the trace entry is replaced by the relative error of one
  // explicit pass over X with FP64 sums (the identity cancels near a good fit).
  ResidualWork<T> rw;
  const bool exact = exact_every > 0 && trace;
  if (exact || rel_err) NNC_TRY(residual_prepare<T>(d, dims, 1, m, r, sc, &rw));
  const T* fac[kMaxD];
  for (int k = 0; k < d; ++k) fac[k] = A[k];
  auto after = [&](int t, cudaStream_t cs) -> int {
    if (exact && ((t + 1) % exact_every == 0 || t + 1 == iters))
      NNC_TRY(residual_run<T>(X, d, dims, 1, m, r, fac, nullptr, rw, nullptr, trace + t, cs));
    return NNC_OK;
  };
  NNC_TRY(replay(iters, s, [&](cudaStream_t cs) -> int {
    NNC_TRY(pass_last(w, A[d - 1], cs));
    for (int n = 0; n < d; ++n) {
      if (n == d - 1) NNC_TRY(pass_first(w, A[0], cs));
      const T* Z = nullptr;
      NNC_TRY(z_chain(w, n, A, &Z, cs));
      NNC_TRY(mttkrp_and_v(w, n, Z, B, cs));
      // Den = A^(n) V_n into gA; MU in place.
      NNC_CUDA_TRY(small_gemm<T>((int)w.N[n], r, r, A[n], r, 1, w.V, r, 1, nullptr, w.gA, cs));
      NNC_CUDA_TRY(launch_elementwise_mu<T>(A[n], w.MT, w.gA, w.N[n] * r, eps, cs));
      NNC_TRY(refresh_a(w, n, A[n], B[n], cs));
      if (n == 0 && d > 2) NNC_TRY(make_u0(w, A[0], cs));
    }
    return loss_into(w, d - 1, last, trace, counter, cs, /*rel=*/1);
  }, after));
  NNC_TRY(check_tc(w, s));
  NNC_TRY(check_trace_finite(counter, s, "nncp_tensor_fit"));
  if (rel_err) {
    if (iters == 0) {
      *rel_err = NAN;
    } else {
      // The final error from an explicit FP64 pass over X, as ntd_fit reports it.
      NNC_TRY(residual_run<T>(X, d, dims, 1, m, r, fac, nullptr, rw, nullptr, last, s));
      NNC_CUDA_TRY(cudaMemcpyAsync(rel_err, last, sizeof(double), cudaMemcpyDeviceToHost, s));
      NNC_CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  return NNC_OK;
}

// NMF A ~ F B (A N x r, F N x m, B m x r) by MU (Alg. 2, second step):
//   F <- max(F .* (A B^T) / max(F (B B^T), eps), 0),
//   B <- max(B .* (F^T A) / max((F^T F) B, eps), 0).
// trace[t] (device, optional) = ||A - F B|| / ||A|| after iteration t.
template <typename T>
int nmf_fit(const T* A, int64_t N, int r, int m, int iters, double eps, T* F, T* B,
            double* trace, double* rel_err, cudaStream_t s) {
  Scratch sc(s);
  T *numF, *denF, *BBt, *numB, *denB, *FtF, *R;
  double *a, *last;
  int* counter;
  NNC_TRY(sc.get(&numF, (size_t)(N * m)));
  NNC_TRY(sc.get(&denF, (size_t)(N * m)));
  NNC_TRY(sc.get(&BBt, (size_t)m * m));
  NNC_TRY(sc.get(&numB, (size_t)m * r));
  NNC_TRY(sc.get(&denB, (size_t)m * r));
  NNC_TRY(sc.get(&FtF, (size_t)m * m));
  NNC_TRY(sc.get(&R, (size_t)(N * r)));
  NNC_TRY(sc.get(&a, 1));
  NNC_TRY(sc.get(&last, 1));
  NNC_TRY(sc.get(&counter, 2));
  NNC_CUDA_TRY(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  rel_norm_kernel<T><<<1, 256, 0, s>>>(A, N * r, nullptr, a, nullptr, nullptr);  // ||A||
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_TRY(replay(iters, s, [&](cudaStream_t cs) -> int {
    NNC_CUDA_TRY(small_gemm<T>((int)N, m, r, A, r, 1, B, 1, r, nullptr, numF, cs));  // A B^T
    NNC_CUDA_TRY(small_gemm<T>(m, m, r, B, r, 1, B, 1, r, nullptr, BBt, cs));        // B B^T
    NNC_CUDA_TRY(small_gemm<T>((int)N, m, m, F, m, 1, BBt, m, 1, nullptr, denF, cs));
    NNC_CUDA_TRY(launch_elementwise_mu<T>(F, numF, denF, N * m, eps, cs));
    NNC_CUDA_TRY(small_gemm<T>(m, r, (int)N, F, 1, m, A, r, 1, nullptr, numB, cs));  // F^T A
    NNC_CUDA_TRY(small_gemm<T>(m, m, (int)N, F, 1, m, F, m, 1, nullptr, FtF, cs));   // F^T F
    NNC_CUDA_TRY(small_gemm<T>(m, r, m, FtF, m, 1, B, r, 1, nullptr, denB, cs));
    NNC_CUDA_TRY(launch_elementwise_mu<T>(B, numB, denB, (int64_t)m * r, eps, cs));
    NNC_CUDA_TRY(small_gemm<T>((int)N, r, m, F, m, 1, B, r, 1, A, R, cs));  // F B - A
    rel_norm_kernel<T><<<1, 256, 0, cs>>>(R, N * r, a, last, trace, counter);
    note_launch(cs);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  }));
  NNC_TRY(check_trace_finite(counter, s, "nmf_fit"));
  if (rel_err) {
    if (iters == 0) {
      *rel_err = NAN;
    } else {
      NNC_CUDA_TRY(cudaMemcpyAsync(rel_err, last, sizeof(double), cudaMemcpyDeviceToHost, s));
      NNC_CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  return NNC_OK;
}


// nnTD of a d-way X (d = 3 or 4) by MU sweeps (Alg. 1, first step), built on
// the mode-product machinery above with F := F^(k). A sweep updates
// F^(1), ..., F^(d), then G:
//   Num_n = unfold_n(Z_n) unfold_n(G)^T           (Z_n from the two passes)
//   H_n   = unfold_n(G x_{k!=n} S_k) unfold_n(G)^T,  S_k = F^(k)T F^(k)
//   F^(n) <- max(F^(n) .* Num_n / max(F^(n) H_n, eps), 0),  S_n refreshed
//   M = Z_d x_d F^(d)T,  D = G x_k S_k,  G <- max(G .* M / max(D, eps), 0)
// and the trace entry sqrt(max(||X||^2 - 2<M, G> + <G, G x_k S_k>, 0)) / ||X||
// in FP64. Z_1 .. Z_{d-1} come from T_last = X x_d F^(d)T (U0 after mode 1)
// and Z_d from T_first = X x_1 F^(1)T formed after mode d-1, so every Z_n sees
// the factors of modes k < n already updated (Gauss-Seidel) and X is read twice
// per sweep. The unfolding products are split-K contractions over the
// flattened (modes before n, modes after n) index.
template <typename T>
int ntd_fit_nway(const T* X, int d, const int64_t* dims, const int* m, bool tensor_cores,
                 int iters, double eps, T* const* F, T* G, double* trace, double* rel_err,
                 cudaStream_t s) {
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  int64_t nc = 1;
  for (int k = 0; k < d; ++k) nc *= m[k];
  Scratch sc(s);
  Work<T> w;
  NNC_TRY(setup(w, X, d, dims, m, /*r=*/1, tensor_cores, sc, s));
  double st[3];
  NNC_CUDA_TRY(cudaMemcpyAsync(st, w.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (st[1] > 0.0) return NNC_ERR_NEGATIVE_INPUT;
  if (!(st[0] > 0.0)) return NNC_ERR_INVALID_ARG;  // X == 0: the relative error is undefined
  int64_t nmax = 1;
  int mmax = 1;
  for (int k = 0; k < d; ++k) {
    nmax = dims[k] > nmax ? dims[k] : nmax;
    mmax = m[k] > mmax ? m[k] : mmax;
  }
  T *num = nullptr, *c0 = nullptr, *c1 = nullptr, *M = nullptr, *D = nullptr;
  T* S[kMaxD] = {};
  double* dummy = nullptr;
  int* counter = nullptr;
  NNC_TRY(sc.get(&num, (size_t)(nmax * mmax)));
  NNC_TRY(sc.get(&c0, (size_t)nc));
  NNC_TRY(sc.get(&c1, (size_t)nc));
  NNC_TRY(sc.get(&M, (size_t)nc));
  NNC_TRY(sc.get(&D, (size_t)nc));
  for (int k = 0; k < d; ++k) NNC_TRY(sc.get(&S[k], (size_t)m[k] * m[k]));
  double* idpart = nullptr;
  NNC_TRY(sc.get(&idpart, 2 * kIdentityBlocks));
  NNC_TRY(sc.get(&dummy, 1));
  NNC_TRY(sc.get(&counter, 2));
  NNC_CUDA_TRY(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
  for (int k = 0; k < d; ++k) NNC_TRY(launch_gram<T>(F[k], dims[k], m[k], S[k], s));
  double* tr = trace ? trace : dummy;
  const int stride = trace ? 1 : 0;
  // The H_n branch (the core times the Grams, then its unfolding product)
  // needs neither Z_n nor the passes, so it runs on a side stream beside the
  // mode products and contractions of Z_n, with split-K scratch of its own.
  // (Leaving the passes SMs for it as well cost more than it saved: 0, 16 and
  // 32 SMs left free gave 713, 748 and 787 us per sweep at 128^3 x 64.)
  T* split2 = nullptr;
  NNC_TRY(sc.get(&split2, w.split_cap));
  SideStream side;
  NNC_TRY(side.init());
  auto fork = [&](cudaStream_t cs) -> int {
    NNC_CUDA_TRY(cudaEventRecord(side.fork, cs));
    NNC_CUDA_TRY(cudaStreamWaitEvent(side.s, side.fork, 0));
    return NNC_OK;
  };
  auto join = [&](cudaStream_t cs) -> int {
    NNC_CUDA_TRY(cudaEventRecord(side.join, side.s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(cs, side.join, 0));
    return NNC_OK;
  };
  // out = G x_k S_k over the modes k != skip (all modes when skip < 0).
  auto core_times_grams = [&](int skip, T* out, T* c0, T* c1, T* split, cudaStream_t cs) -> int {
    const T* src = G;
    int left = 0;
    for (int k = 0; k < d; ++k) left += k != skip;
    for (int k = 0; k < d; ++k) {
      if (k == skip) continue;
      T* dst = --left == 0 ? out : (src == c0 ? c1 : c0);
      int64_t pre = 1, post = 1;
      for (int j = 0; j < k; ++j) pre *= m[j];
      for (int j = k + 1; j < d; ++j) post *= m[j];
      NNC_CUDA_TRY(launch_ttm<T>(src, pre, m[k], post, S[k], m[k], 1, m[k], dst, split,
                                 w.split_cap, cs));
      src = dst;
    }
    return NNC_OK;
  };
  // H_n = unfold_n(G x_{k!=n} S_k) unfold_n(G)^T on the side stream, formed in
  // M (free until the core update).
  auto h_branch = [&](int n) -> int {
    int64_t pre = 1, post = 1;
    for (int j = 0; j < n; ++j) pre *= m[j];
    for (int j = n + 1; j < d; ++j) post *= m[j];
    NNC_TRY(core_times_grams(n, M, c0, c1, split2, side.s));
    NNC_CUDA_TRY(launch_pair_contract<T>(M, G, pre, m[n], m[n], post, w.H, split2, w.split_cap,
                                         side.s));
    return NNC_OK;
  };
  // The core update of a sweep (M = Z_d x_d F^(d)T with the updated F^(d),
  // D = G x_k S_k, the MU step on G, then G x_k S_k of the new core and the
  // trace entry) needs neither the next sweep's pass X x_d F^(d)T nor its Z_1
  // chain, so it runs on the side stream at the start of the next sweep,
  // beside them (m_ready: M is formed, so Z_d's buffer may be reused; g_ready:
  // the new G, which Num_1 needs); the last sweep's runs after the replays.
  // Each step is the same launch as in a sweep that ends with its own core
  // update, so the results are the same.
  const T* zlast = nullptr;  // Z_d of the sweep whose core update is pending
  auto core_update = [&](cudaStream_t cs, T* split, bool mark) -> int {
    const int64_t lead = nc / m[d - 1];
    NNC_CUDA_TRY(launch_ttm<T>(zlast, lead, (int)dims[d - 1], 1, F[d - 1], m[d - 1], 1,
                               m[d - 1], M, split, w.split_cap, cs));
    if (mark) NNC_CUDA_TRY(cudaEventRecord(side.m_ready, cs));
    NNC_TRY(core_times_grams(-1, D, c0, c1, split, cs));
    NNC_CUDA_TRY(launch_elementwise_mu<T>(G, M, D, nc, eps, cs));
    if (mark) NNC_CUDA_TRY(cudaEventRecord(side.g_ready, cs));
    NNC_TRY(core_times_grams(-1, D, c0, c1, split, cs));
    NNC_CUDA_TRY(
        launch_residual_identity<T>(M, G, D, nc, w.stats, tr, stride, counter, idpart, cs));
    return NNC_OK;
  };
  auto sweep = [&](cudaStream_t cs, bool pending) -> int {
    const T* Z = nullptr;
    for (int n = 0; n < d; ++n) {
      // H_n beside Z_n, forked after the previous mode's Gram (mode 1: after
      // the previous sweep's core update).
      NNC_TRY(fork(cs));
      if (n == 0 && pending) NNC_TRY(core_update(side.s, split2, true));
      NNC_TRY(h_branch(n));
      if (n == 0) NNC_TRY(pass_last(w, F[d - 1], cs));
      if (n == d - 1) NNC_TRY(pass_first(w, F[0], cs));
      if (n == 0 && pending) NNC_CUDA_TRY(cudaStreamWaitEvent(cs, side.m_ready, 0));
      NNC_TRY(z_chain(w, n, F, &Z, cs));
      if (n == 0 && pending) NNC_CUDA_TRY(cudaStreamWaitEvent(cs, side.g_ready, 0));
      int64_t pre = 1, post = 1;
      for (int j = 0; j < n; ++j) pre *= m[j];
      for (int j = n + 1; j < d; ++j) post *= m[j];
      // Num_n's split partials are added by the MU kernel (in split order).
      int parts = 1;
      NNC_CUDA_TRY(launch_pair_contract<T>(Z, G, pre, (int)dims[n], m[n], post, num, w.split,
                                           w.split_cap, cs, &parts));
      NNC_TRY(join(cs));
      NNC_CUDA_TRY(launch_factor_mu<T>(F[n], parts > 1 ? w.split : num, w.H, dims[n], m[n], eps,
                                       cs, parts));
      NNC_TRY(launch_gram<T>(F[n], dims[n], m[n], S[n], cs));
      if (n == 0 && d > 2) NNC_TRY(make_u0(w, F[0], cs));
    }
    zlast = Z;
    return NNC_OK;
  };
  NNC_TRY(replay_pipelined(
      iters, s, [&](cudaStream_t cs) -> int { return sweep(cs, false); },
      [&](cudaStream_t cs) -> int { return sweep(cs, true); },
      [&](cudaStream_t cs) -> int { return core_update(cs, w.split, false); }));
  NNC_TRY(check_tc(w, s));
  NNC_TRY(check_trace_finite(counter, s, "ntd_fit"));
  if (rel_err) {
    double* out2 = nullptr;
    NNC_TRY(sc.get(&out2, 2));
    const T* fac[kMaxD];
    for (int k = 0; k < d; ++k) fac[k] = F[k];
    NNC_TRY(residual_device<T>(X, d, dims, 0, m, 0, fac, G, out2, sc, s));
    double h[2];
    NNC_CUDA_TRY(cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, s));
    NNC_CUDA_TRY(cudaStreamSynchronize(s));
    *rel_err = sqrt(h[0] / h[1]);
  }
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  return NNC_OK;
}

template int lifted_grad<float>(const float*, int, const int64_t*, const int*, int, bool,
                                float* const*, float* const*, float* const*, float* const*,
                                double*, cudaStream_t);
template int lifted_grad<double>(const double*, int, const int64_t*, const int*, int, bool,
                                 double* const*, double* const*, double* const*, double* const*,
                                 double*, cudaStream_t);
template int lifted_pg_fit<float>(const float*, int, const int64_t*, const int*, int, bool, int,
                                  float* const*, float* const*, double*, double*, cudaStream_t);
template int nncp_tensor_fit<float>(const float*, int, const int64_t*, int, bool, int, double, int,
                                    float* const*, double*, double*, cudaStream_t);
template int nncp_tensor_fit<double>(const double*, int, const int64_t*, int, bool, int, double, int,
                                     double* const*, double*, double*, cudaStream_t);
template int nmf_fit<float>(const float*, int64_t, int, int, int, double, float*, float*,
                            double*, double*, cudaStream_t);
template int nmf_fit<double>(const double*, int64_t, int, int, int, double, double*, double*,
                             double*, double*, cudaStream_t);
template int lifted_pg_fit<double>(const double*, int, const int64_t*, const int*, int, bool,
                                   int, double* const*, double* const*, double*, double*,
                                   cudaStream_t);
template int ntd_fit_nway<float>(const float*, int, const int64_t*, const int*, bool, int, double,
                                 float* const*, float*, double*, double*, cudaStream_t);
template int ntd_fit_nway<double>(const double*, int, const int64_t*, const int*, bool, int,
                                  double, double* const*, double*, double*, double*,
                                  cudaStream_t);

}  // namespace nnc
