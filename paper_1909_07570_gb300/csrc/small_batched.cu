// Batched fits of tiny problems, one thread block per problem, everything in
// shared memory: the workload of the multirank study (Sec. 4.3, Ex. "equal":
// a 4 x 4 x 4 tensor decomposed from many random starts at several
// multiranks) and of many-small-tensor batches.
//
//   ntd_small_kernel     nnTD of a 3-way X (Alg. 1, step 1) by the MU sweep of
//                        ntd_fit: F^(1), F^(2), F^(3), then G;
//   nmf_small_kernel     NMF A ~ F B of one CP factor (Alg. 2, step 2) by MU;
//   lifted_err_kernel    ||X - I x_k F^(k) B^(k)|| / ||X|| of a fitted pair.
//
// Every contraction is a plain loop over shared-memory arrays spread over the
// block's threads, reduced in a fixed order. The jobs' descriptors are copied
// to the device by the call.
#include <vector>

#include "autotune.cuh"
#include "nncp.cuh"
#include "small_batched.cuh"

namespace nnc {
namespace {

constexpr int kThreads = 256;

// out = in x_k A for a 3-way `in` (dims d[0..2], C order): out has d[k]
// replaced by P and out[.., p, ..] = sum_j A[p sp + j sj] in[.., j, ..]. The
// tensor is viewed as (L, J, C) around mode k; j runs in order.
template <typename T>
__device__ void mp3(const T* in, const int* d, int k, const T* A, int sp, int sj, int P, T* out) {
  const int L = k == 0 ? 1 : (k == 1 ? d[0] : d[0] * d[1]);
  const int C = k == 2 ? 1 : (k == 1 ? d[2] : d[1] * d[2]);
  const int J = d[k];
  const int n = L * P * C;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int c = e % C, lp = e / C, p = lp % P, l = lp / P;
    const T* x = in + l * J * C + c;
    const T* a = A + p * sp;
    T s = T(0);
    for (int j = 0; j < J; ++j) s = fma(a[j * sj], x[j * C], s);
    out[e] = s;
  }
  __syncthreads();
}

// out[i, a] = sum over the other two indices of Y[.., i, ..] G[.., a, ..]
// (unfold_n(Y) unfold_n(G)^T); Y has dims dy, G has dims dg, equal off mode n.
// Both are viewed as (L, mode n, C); the terms run over l, then c, in order.
template <typename T>
__device__ void unfold_dot(const T* Y, const int* dy, const T* G, const int* dg, int n, T* out) {
  const int NI = dy[n], MA = dg[n];
  const int L = n == 0 ? 1 : (n == 1 ? dy[0] : dy[0] * dy[1]);
  const int C = n == 2 ? 1 : (n == 1 ? dy[2] : dy[1] * dy[2]);
  for (int e = threadIdx.x; e < NI * MA; e += blockDim.x) {
    const int i = e / MA, a = e % MA;
    T s = T(0);
    for (int l = 0; l < L; ++l) {
      const T* y = Y + (l * NI + i) * C;
      const T* g = G + (l * MA + a) * C;
      for (int c = 0; c < C; ++c) s = fma(y[c], g[c], s);
    }
    out[e] = s;
  }
  __syncthreads();
}

// C (M x N) = sum_k A(i, k) B(k, j), element (i, k) of A at A[i as_i + k as_k].
template <typename T>
__device__ void sgemm(int M, int N, int K, const T* A, int as_i, int as_k, const T* B, int bs_k,
                      int bs_j, T* C) {
  for (int e = threadIdx.x; e < M * N; e += blockDim.x) {
    const int i = e / N, j = e % N;
    T s = T(0);
    for (int k = 0; k < K; ++k) s = fma(A[i * as_i + k * as_k], B[k * bs_k + j * bs_j], s);
    C[e] = s;
  }
  __syncthreads();
}

template <typename T>
__device__ void mu(T* theta, const T* num, const T* den, int n, T eps) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const T v = theta[e] * num[e] / (den[e] > eps ? den[e] : eps);
    theta[e] = v > T(0) ? v : T(0);
  }
  __syncthreads();
}

template <typename T>
__device__ void load(T* dst, const T* src, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

template <typename T>
__device__ void store(T* dst, const T* src, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

// sum (a - b)^2 and sum a^2 in FP64 over n entries (b may be null: 0), in an
// order that does not depend on the block size (`red`: 2 kFixedLanes doubles).
template <typename T>
__device__ void diff_norms(const T* a, const T* b, int n, double* red, double* out2) {
  const double2 r = fixed_sums2(n, [&](int64_t e) {
    const double av = (double)a[e], bv = b ? (double)b[e] : 0.0;
    return make_double2((av - bv) * (av - bv), av * av);
  }, red);
  if (threadIdx.x == 0) {
    out2[0] = r.x;
    out2[1] = r.y;
  }
  __syncthreads();
}

size_t ntd_small_elems(const ntd_small_job& j) {
  size_t big = 1, nx = 1, ng = 1, f = 0, s = 0, nm = 0, mm = 0;
  for (int k = 0; k < 3; ++k) {
    const int mk = j.m[k], nk = j.dims[k];
    big *= (size_t)(mk > nk ? mk : nk);
    nx *= nk;
    ng *= mk;
    f += (size_t)nk * mk;
    s += (size_t)mk * mk;
    nm = (size_t)nk * mk > nm ? (size_t)nk * mk : nm;
    mm = (size_t)mk * mk > mm ? (size_t)mk * mk : mm;
  }
  return nx + f + ng + s + 2 * big + 2 * nm + mm + 2 * ng;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
ntd_small_kernel(const ntd_small_job* __restrict__ jobs, int iters, T eps, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double nrm[2];
  const ntd_small_job& jb = jobs[blockIdx.x];
  const int* N = jb.dims;
  const int* m = jb.m;
  const int nx = N[0] * N[1] * N[2], ng = m[0] * m[1] * m[2];
  int big = 1, nm = 0, mm = 0;
  for (int k = 0; k < 3; ++k) {
    big *= m[k] > N[k] ? m[k] : N[k];
    nm = N[k] * m[k] > nm ? N[k] * m[k] : nm;
    mm = m[k] * m[k] > mm ? m[k] * m[k] : mm;
  }
  T* X = reinterpret_cast<T*>(smem_raw);
  T* F[3];
  F[0] = X + nx;
  F[1] = F[0] + N[0] * m[0];
  F[2] = F[1] + N[1] * m[1];
  T* G = F[2] + N[2] * m[2];
  T* S[3];
  S[0] = G + ng;
  S[1] = S[0] + m[0] * m[0];
  S[2] = S[1] + m[1] * m[1];
  T* t1 = S[2] + m[2] * m[2];
  T* t2 = t1 + big;
  T* num = t2 + big;
  T* den = num + nm;
  T* H = den + nm;
  T* M = H + mm;
  T* D = M + ng;
  load(X, static_cast<const T*>(jb.X), nx);
  for (int k = 0; k < 3; ++k) load(F[k], static_cast<const T*>(jb.F[k]), N[k] * m[k]);
  load(G, static_cast<const T*>(jb.G), ng);
  __syncthreads();
  for (int k = 0; k < 3; ++k) sgemm(m[k], m[k], N[k], F[k], 1, m[k], F[k], m[k], 1, S[k]);

  for (int it = 0; it < iters; ++it) {
    for (int n = 0; n < 3; ++n) {
      // Z = X x_{k!=n} F_k^T (into t1 or t2), Num = unfold_n(Z) unfold_n(G)^T
      int dz[3] = {N[0], N[1], N[2]};
      const T* src = X;
      T* bufs[2] = {t1, t2};
      int b = 0;
      for (int k = 0; k < 3; ++k) {
        if (k == n) continue;
        mp3(src, dz, k, F[k], 1, m[k], m[k], bufs[b]);
        dz[k] = m[k];
        src = bufs[b];
        b ^= 1;
      }
      unfold_dot(src, dz, G, m, n, num);
      // W = G x_{k!=n} S_k, H = unfold_n(W) unfold_n(G)^T, Den = F_n H
      int dw[3] = {m[0], m[1], m[2]};
      src = G;
      for (int k = 0; k < 3; ++k) {
        if (k == n) continue;
        mp3(src, dw, k, S[k], m[k], 1, m[k], bufs[b]);
        src = bufs[b];
        b ^= 1;
      }
      unfold_dot(src, dw, G, m, n, H);
      sgemm(N[n], m[n], m[n], F[n], m[n], 1, H, m[n], 1, den);
      mu(F[n], num, den, N[n] * m[n], eps);
      sgemm(m[n], m[n], N[n], F[n], 1, m[n], F[n], m[n], 1, S[n]);
    }
    // Core: M = X x_k F_k^T, D = G x_k S_k
    int dz[3] = {N[0], N[1], N[2]};
    mp3(X, dz, 0, F[0], 1, m[0], m[0], t1);
    dz[0] = m[0];
    mp3(t1, dz, 1, F[1], 1, m[1], m[1], t2);
    dz[1] = m[1];
    mp3(t2, dz, 2, F[2], 1, m[2], m[2], M);
    int dg[3] = {m[0], m[1], m[2]};
    mp3(G, dg, 0, S[0], m[0], 1, m[0], t1);
    mp3(t1, dg, 1, S[1], m[1], 1, m[1], t2);
    mp3(t2, dg, 2, S[2], m[2], 1, m[2], D);
    mu(G, M, D, ng, eps);
  }
  // ||X - G x_k F_k|| / ||X|| by brute force
  int dr[3] = {m[0], m[1], m[2]};
  mp3(G, dr, 0, F[0], m[0], 1, N[0], t1);
  dr[0] = N[0];
  mp3(t1, dr, 1, F[1], m[1], 1, N[1], t2);
  dr[1] = N[1];
  mp3(t2, dr, 2, F[2], m[2], 1, N[2], t1);
  diff_norms(X, t1, nx, red, nrm);
  if (threadIdx.x == 0 && rel_errs) rel_errs[blockIdx.x] = sqrt(nrm[0] / nrm[1]);
  for (int k = 0; k < 3; ++k) store(static_cast<T*>(jb.F[k]), F[k], N[k] * m[k]);
  store(static_cast<T*>(jb.G), G, ng);
}

// ---- problems whose X does not fit in shared memory -------------------------
//
// One thread block per problem as above, but X stays in global memory (with
// two blocks per SM in flight, their tensors stay in L2) and a sweep reads it
// twice, like ntd_fit: P3 = X x_3 F^(3)T serves modes 1 and 2, P1 = X x_1
// F^(1)T (new F^(1)) mode 3 and the core. Factors, core, Grams and pass
// results live in shared memory.

// acc[p] += v f[p] for p < Q (Q <= QM); with vec, f is 16-byte aligned and
// Q % 4 == 0, and the factor row comes in 16-byte shared loads (a warp reads
// the same row: one broadcast per load), four times fewer loads than the FMAs
// would issue one by one.
template <typename T, int QM>
__device__ __forceinline__ void axpy_row(T v, const T* f, int Q, bool vec, T (&acc)[QM]) {
  if (vec) {
#pragma unroll
    for (int p = 0; p < QM; p += 4) {
      if (p < Q) {
        T w[4];
        if constexpr (sizeof(T) == 4) {
          const float4 t = *reinterpret_cast<const float4*>(f + p);
          w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
        } else {
          const double2 a = *reinterpret_cast<const double2*>(f + p);
          const double2 b = *reinterpret_cast<const double2*>(f + p + 2);
          w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[p + u] = fma(v, w[u], acc[p + u]);
      }
    }
  } else {
#pragma unroll
    for (int p = 0; p < QM; ++p)
      if (p < Q) acc[p] = fma(v, f[p], acc[p]);
  }
}

// P[r, p] = sum_k X[r N3 + k] F[k, p], rows r < R of X viewed R x N3, p < Q
// (F: N3 x Q in shared memory). One thread per row, Q accumulators; the rows
// a warp walks share their L1 lines.
template <typename T, int QM, bool VEC>
__device__ void pass_rows_impl(const T* __restrict__ X, int R, int N3, const T* F, int Q, T* P) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    T acc[QM];
#pragma unroll
    for (int p = 0; p < QM; ++p) acc[p] = T(0);
    const T* x = X + (int64_t)r * N3;
    int k = 0;
    for (; k + 8 <= N3; k += 8) {  // 8 loads in flight, then the terms in order
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(x + k + u);
#pragma unroll
      for (int u = 0; u < 8; ++u) axpy_row<T, QM>(v[u], F + (k + u) * Q, Q, VEC, acc);
    }
    for (; k < N3; ++k) axpy_row<T, QM>(__ldg(x + k), F + k * Q, Q, VEC, acc);
#pragma unroll
    for (int p = 0; p < QM; ++p)
      if (p < Q) P[r * Q + p] = acc[p];
  }
  __syncthreads();
}

template <typename T, int QM>
__device__ void pass_rows(const T* __restrict__ X, int R, int N3, const T* F, int Q, T* P) {
  if ((Q & 3) == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0)
    pass_rows_impl<T, QM, true>(X, R, N3, F, Q, P);
  else
    pass_rows_impl<T, QM, false>(X, R, N3, F, Q, P);
}

// P[p, c] = sum_i F[i, p] X[i C + c], X viewed N1 x C (F: N1 x Q in shared
// memory). One thread per column c: consecutive threads read consecutive c.
template <typename T, int QM, bool VEC>
__device__ void pass_cols_impl(const T* __restrict__ X, int N1, int C, const T* F, int Q, T* P) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    T acc[QM];
#pragma unroll
    for (int p = 0; p < QM; ++p) acc[p] = T(0);
    int i = 0;
    for (; i + 8 <= N1; i += 8) {  // 8 loads in flight, then the terms in order
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldg(X + (int64_t)(i + u) * C + c);
#pragma unroll
      for (int u = 0; u < 8; ++u) axpy_row<T, QM>(v[u], F + (i + u) * Q, Q, VEC, acc);
    }
    for (; i < N1; ++i) axpy_row<T, QM>(__ldg(X + (int64_t)i * C + c), F + i * Q, Q, VEC, acc);
#pragma unroll
    for (int p = 0; p < QM; ++p)
      if (p < Q) P[(int64_t)p * C + c] = acc[p];
  }
  __syncthreads();
}

template <typename T, int QM>
__device__ void pass_cols(const T* __restrict__ X, int N1, int C, const T* F, int Q, T* P) {
  if ((Q & 3) == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0)
    pass_cols_impl<T, QM, true>(X, N1, C, F, Q, P);
  else
    pass_cols_impl<T, QM, false>(X, N1, C, F, Q, P);
}

// sum (X - X_hat)^2 and sum X^2 in FP64 with X_hat[r, k] = sum_c U[r, c] W[k, c]
// (X viewed R x N3 in global memory, U: R x K and W: N3 x K in shared memory).
template <typename T>
__device__ void stream_residual(const T* __restrict__ X, int R, int N3, const T* U, const T* W,
                                int K, double* red, double* out2) {
  const double2 r2 = fixed_sums2((int64_t)R * N3, [&](int64_t e) {
    const int r = (int)(e / N3), k = (int)(e - (int64_t)r * N3);
    T h = T(0);
    for (int c = 0; c < K; ++c) h = fma(U[r * K + c], W[k * K + c], h);
    const double xv = (double)__ldg(X + e), dv = xv - (double)h;
    return make_double2(dv * dv, xv * xv);
  }, red);
  if (threadIdx.x == 0) {
    out2[0] = r2.x;
    out2[1] = r2.y;
  }
  __syncthreads();
}

struct NtdL2Sizes {
  int p, y, nm, mm, ng;
};

__host__ __device__ inline NtdL2Sizes ntd_l2_sizes(const int* N, const int* m) {
  NtdL2Sizes z;
  const int p3 = N[0] * N[1] * m[2], p1 = m[0] * N[1] * N[2];
  z.p = p3 > p1 ? p3 : p1;
  const int y1 = N[0] * m[1] * m[2], y2 = m[0] * N[1] * m[2], y3 = m[0] * m[1] * N[2];
  z.y = y1 > y2 ? (y1 > y3 ? y1 : y3) : (y2 > y3 ? y2 : y3);
  z.nm = 0;
  z.mm = 0;
  for (int k = 0; k < 3; ++k) {
    z.nm = N[k] * m[k] > z.nm ? N[k] * m[k] : z.nm;
    z.mm = m[k] * m[k] > z.mm ? m[k] * m[k] : z.mm;
  }
  z.ng = m[0] * m[1] * m[2];
  return z;
}

size_t ntd_l2_elems(const ntd_small_job& j) {
  const NtdL2Sizes z = ntd_l2_sizes(j.dims, j.m);
  size_t f = 0, s = 0;
  for (int k = 0; k < 3; ++k) {
    f += (size_t)j.dims[k] * j.m[k];
    s += (size_t)j.m[k] * j.m[k];
  }
  return f + s + (size_t)z.p + z.y + 2 * (size_t)z.nm + z.mm + 4 * (size_t)z.ng;
}

// nnTD of one job per block with X in global memory: the sweep of ntd_fit,
// F^(1), F^(2), F^(3) by MU (Num_n from the pass results, H_n from the core
// and the Grams), then G with M = Y3 x_3 F^(3)T and D = (G x_1 S1 x_2 S2) x_3
// S3; the final relative error by one more stream over X.
template <typename T, int QM>
__global__ void __launch_bounds__(kThreads, 2)
ntd_l2_kernel(const ntd_small_job* __restrict__ jobs, int iters, T eps, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double nrm[2];
  const ntd_small_job& jb = jobs[blockIdx.x];
  const int* N = jb.dims;
  const int* m = jb.m;
  const T* X = static_cast<const T*>(jb.X);
  const NtdL2Sizes z = ntd_l2_sizes(N, m);
  T* F[3];
  F[0] = reinterpret_cast<T*>(smem_raw);
  F[1] = F[0] + N[0] * m[0];
  F[2] = F[1] + N[1] * m[1];
  T* G = F[2] + N[2] * m[2];
  T* S[3];
  S[0] = G + z.ng;
  S[1] = S[0] + m[0] * m[0];
  S[2] = S[1] + m[1] * m[1];
  T* P = S[2] + m[2] * m[2];
  T* Y = P + z.p;
  T* num = Y + z.y;
  T* den = num + z.nm;
  T* H = den + z.nm;
  T* W = H + z.mm;
  T* W2 = W + z.ng;
  T* M = W2 + z.ng;
  for (int k = 0; k < 3; ++k) load(F[k], static_cast<const T*>(jb.F[k]), N[k] * m[k]);
  load(G, static_cast<const T*>(jb.G), z.ng);
  __syncthreads();
  for (int k = 0; k < 3; ++k) sgemm(m[k], m[k], N[k], F[k], 1, m[k], F[k], m[k], 1, S[k]);

  const int d3[3] = {N[0], N[1], m[2]};   // P3
  const int d1[3] = {m[0], N[1], N[2]};   // P1
  const int y1[3] = {N[0], m[1], m[2]};
  const int y2[3] = {m[0], N[1], m[2]};
  const int y3[3] = {m[0], m[1], N[2]};
  for (int it = 0; it < iters; ++it) {
    pass_rows<T, QM>(X, N[0] * N[1], N[2], F[2], m[2], P);  // P3 = X x_3 F3^T
    // Mode 1: Num1 from Y1 = P3 x_2 F2^T, H1 from G x_2 S2 x_3 S3.
    mp3(P, d3, 1, F[1], 1, m[1], m[1], Y);
    unfold_dot(Y, y1, G, m, 0, num);
    mp3(G, m, 1, S[1], m[1], 1, m[1], W);
    mp3(W, m, 2, S[2], m[2], 1, m[2], W2);
    unfold_dot(W2, m, G, m, 0, H);
    sgemm(N[0], m[0], m[0], F[0], m[0], 1, H, m[0], 1, den);
    mu(F[0], num, den, N[0] * m[0], eps);
    sgemm(m[0], m[0], N[0], F[0], 1, m[0], F[0], m[0], 1, S[0]);
    // Mode 2: Y2 = P3 x_1 F1^T (new F1), H2 from G x_1 S1 x_3 S3.
    mp3(P, d3, 0, F[0], 1, m[0], m[0], Y);
    unfold_dot(Y, y2, G, m, 1, num);
    mp3(G, m, 0, S[0], m[0], 1, m[0], W);
    mp3(W, m, 2, S[2], m[2], 1, m[2], W2);
    unfold_dot(W2, m, G, m, 1, H);
    sgemm(N[1], m[1], m[1], F[1], m[1], 1, H, m[1], 1, den);
    mu(F[1], num, den, N[1] * m[1], eps);
    sgemm(m[1], m[1], N[1], F[1], 1, m[1], F[1], m[1], 1, S[1]);
    // Mode 3: P1 = X x_1 F1^T, Y3 = P1 x_2 F2^T, H3 from W2 = G x_1 S1 x_2 S2.
    pass_cols<T, QM>(X, N[0], N[1] * N[2], F[0], m[0], P);
    mp3(P, d1, 1, F[1], 1, m[1], m[1], Y);
    unfold_dot(Y, y3, G, m, 2, num);
    mp3(G, m, 0, S[0], m[0], 1, m[0], W);
    mp3(W, m, 1, S[1], m[1], 1, m[1], W2);
    unfold_dot(W2, m, G, m, 2, H);
    sgemm(N[2], m[2], m[2], F[2], m[2], 1, H, m[2], 1, den);
    mu(F[2], num, den, N[2] * m[2], eps);
    sgemm(m[2], m[2], N[2], F[2], 1, m[2], F[2], m[2], 1, S[2]);
    // Core: M = Y3 x_3 F3^T, D = W2 x_3 S3.
    mp3(Y, y3, 2, F[2], 1, m[2], m[2], M);
    mp3(W2, m, 2, S[2], m[2], 1, m[2], W);
    mu(G, M, W, z.ng, eps);
  }
  // ||X - G x_k F_k|| / ||X||: U = G x_1 F1 x_2 F2 (N1, N2, m3), then X streamed.
  const int dg[3] = {m[0], m[1], m[2]};
  mp3(G, dg, 0, F[0], m[0], 1, N[0], Y);
  mp3(Y, y1, 1, F[1], m[1], 1, N[1], P);
  stream_residual(X, N[0] * N[1], N[2], P, F[2], m[2], red, nrm);
  if (threadIdx.x == 0 && rel_errs) rel_errs[blockIdx.x] = sqrt(nrm[0] / nrm[1]);
  for (int k = 0; k < 3; ++k) store(static_cast<T*>(jb.F[k]), F[k], N[k] * m[k]);
  store(static_cast<T*>(jb.G), G, z.ng);
}

// nnCPD of a 3-way tensor per block with the tensor in global memory (the
// sweep of nncp_core_fit: A^(n) <- MU(A^(n), MT_n, A^(n) V_n) for n = 1, 2, 3),
// MT_n from two passes: T = X x_3 A3^T gives MT_1[i, q] = sum_j T[i, j, q]
// A2[j, q] and MT_2[j, q] = sum_i T[i, j, q] A1[i, q] (new A1); T' = X x_1
// A1^T gives MT_3[k, q] = sum_j T'[q, j, k] A2[j, q] (new A2).

template <typename T, int QM>
__global__ void __launch_bounds__(kThreads, 2)
cpx_l2_kernel(const nncp_job* __restrict__ jobs, int iters, T eps, double* rel_errs,
              int* statuses) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double nrm[2];
  const nncp_job& jb = jobs[blockIdx.x];
  // A job the host skipped (its shared memory was not sized for it).
  if (!nncp_job_valid(jb) || jb.d != 3) {
    if (statuses != nullptr && threadIdx.x == 0) statuses[blockIdx.x] = NNC_ERR_INVALID_ARG;
    return;
  }
  const int* N = jb.m;
  const int r = jb.r;
  const T* X = static_cast<const T*>(jb.G);
  int nmax = N[0] > N[1] ? N[0] : N[1];
  nmax = nmax > N[2] ? nmax : N[2];
  const int t3 = N[0] * N[1] * r, t1 = r * N[1] * N[2];
  T* A[3];
  A[0] = reinterpret_cast<T*>(smem_raw);
  A[1] = A[0] + N[0] * r;
  A[2] = A[1] + N[1] * r;
  T* Gr[3];
  Gr[0] = A[2] + N[2] * r;
  Gr[1] = Gr[0] + r * r;
  Gr[2] = Gr[1] + r * r;
  T* Tb = Gr[2] + r * r;
  T* MT = Tb + (t3 > t1 ? t3 : t1);
  T* den = MT + nmax * r;
  T* V = den + nmax * r;
  for (int k = 0; k < 3; ++k) load(A[k], static_cast<const T*>(jb.B[k]), N[k] * r);
  __syncthreads();
  for (int k = 0; k < 3; ++k) sgemm(r, r, N[k], A[k], 1, r, A[k], r, 1, Gr[k]);
  // V = Gr[a] .* Gr[b], den = A[n] V, MU on A[n], Gram of the new A[n].
  auto update = [&](int n, int a, int b) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) V[e] = Gr[a][e] * Gr[b][e];
    __syncthreads();
    sgemm(N[n], r, r, A[n], r, 1, V, r, 1, den);
    mu(A[n], MT, den, N[n] * r, eps);
    sgemm(r, r, N[n], A[n], 1, r, A[n], r, 1, Gr[n]);
  };
  for (int it = 0; it < iters; ++it) {
    pass_rows<T, QM>(X, N[0] * N[1], N[2], A[2], r, Tb);  // T[i, j, q]
    for (int e = threadIdx.x; e < N[0] * r; e += blockDim.x) {
      const int i = e / r, q = e - i * r;
      T acc = T(0);
      for (int j = 0; j < N[1]; ++j) acc = fma(Tb[(i * N[1] + j) * r + q], A[1][j * r + q], acc);
      MT[e] = acc;
    }
    __syncthreads();
    update(0, 1, 2);
    for (int e = threadIdx.x; e < N[1] * r; e += blockDim.x) {
      const int j = e / r, q = e - j * r;
      T acc = T(0);
      for (int i = 0; i < N[0]; ++i) acc = fma(Tb[(i * N[1] + j) * r + q], A[0][i * r + q], acc);
      MT[e] = acc;
    }
    __syncthreads();
    update(1, 0, 2);
    pass_cols<T, QM>(X, N[0], N[1] * N[2], A[0], r, Tb);  // T'[q, j, k]
    for (int e = threadIdx.x; e < N[2] * r; e += blockDim.x) {
      const int k = e / r, q = e - k * r;
      T acc = T(0);
      for (int j = 0; j < N[1]; ++j)
        acc = fma(Tb[(q * N[1] + j) * N[2] + k], A[1][j * r + q], acc);
      MT[e] = acc;
    }
    __syncthreads();
    update(2, 0, 1);
  }
  // ||X - I x_k A_k|| / ||X||: U[i, j, q] = A1[i, q] A2[j, q], then X streamed.
  for (int e = threadIdx.x; e < t3; e += blockDim.x) {
    const int q = e % r, ij = e / r, j = ij % N[1], i = ij / N[1];
    Tb[e] = A[0][i * r + q] * A[1][j * r + q];
  }
  __syncthreads();
  stream_residual(X, N[0] * N[1], N[2], Tb, A[2], r, red, nrm);
  if (threadIdx.x == 0 && rel_errs) rel_errs[blockIdx.x] = sqrt(nrm[0] / nrm[1]);
  for (int k = 0; k < 3; ++k) store(static_cast<T*>(jb.B[k]), A[k], N[k] * r);
  if (statuses != nullptr) {
    // NONFINITE when a NaN or an overflow shows in the factors or the sums.
    bool finite = true;
    for (int k = 0; k < 3; ++k)
      for (int e = threadIdx.x; e < N[k] * r; e += blockDim.x) finite = finite && isfinite(A[k][e]);
    const int ok = __syncthreads_and(finite ? 1 : 0);
    if (threadIdx.x == 0)
      statuses[blockIdx.x] =
          (ok && isfinite(nrm[0]) && isfinite(nrm[1])) ? NNC_OK : NNC_ERR_NONFINITE;
  }
}

size_t nmf_small_elems(const nmf_job& j) {
  const size_t N = j.N, r = j.r, m = j.m;
  return N * r + N * m + m * r + 2 * m * m + 2 * N * m + 2 * m * r + N * r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
nmf_small_kernel(const nmf_job* __restrict__ jobs, int iters, T eps, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double nrm[2];
  const nmf_job& jb = jobs[blockIdx.x];
  const int N = jb.N, r = jb.r, m = jb.m;
  T* A = reinterpret_cast<T*>(smem_raw);
  T* F = A + N * r;
  T* B = F + N * m;
  T* BBt = B + m * r;
  T* FtF = BBt + m * m;
  T* numF = FtF + m * m;
  T* denF = numF + N * m;
  T* numB = denF + N * m;
  T* denB = numB + m * r;
  T* R = denB + m * r;
  load(A, static_cast<const T*>(jb.A), N * r);
  load(F, static_cast<T*>(jb.F), N * m);
  load(B, static_cast<T*>(jb.B), m * r);
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    sgemm(N, m, r, A, r, 1, B, 1, r, numF);       // A B^T
    sgemm(m, m, r, B, r, 1, B, 1, r, BBt);        // B B^T
    sgemm(N, m, m, F, m, 1, BBt, m, 1, denF);     // F (B B^T)
    mu(F, numF, denF, N * m, eps);
    sgemm(m, r, N, F, 1, m, A, r, 1, numB);       // F^T A
    sgemm(m, m, N, F, 1, m, F, m, 1, FtF);        // F^T F
    sgemm(m, r, m, FtF, m, 1, B, r, 1, denB);     // (F^T F) B
    mu(B, numB, denB, m * r, eps);
  }
  sgemm(N, r, m, F, m, 1, B, r, 1, R);
  diff_norms(A, R, N * r, red, nrm);
  if (threadIdx.x == 0 && rel_errs) rel_errs[blockIdx.x] = sqrt(nrm[0] / nrm[1]);
  store(static_cast<T*>(jb.F), F, N * m);
  store(static_cast<T*>(jb.B), B, m * r);
}

size_t lifted_small_elems(const lifted_job& j) {
  size_t a = 0;
  for (int k = 0; k < 3; ++k) a += (size_t)j.dims[k] * j.r;
  return a;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
lifted_err_kernel(const lifted_job* __restrict__ jobs, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double nrm[2];
  const lifted_job& jb = jobs[blockIdx.x];
  const int* N = jb.dims;
  const int r = jb.r;
  T* A[3];
  A[0] = reinterpret_cast<T*>(smem_raw);
  A[1] = A[0] + N[0] * r;
  A[2] = A[1] + N[1] * r;
  for (int k = 0; k < 3; ++k)  // A_k = F_k B_k
    sgemm(N[k], r, jb.m[k], static_cast<const T*>(jb.F[k]), jb.m[k], 1,
          static_cast<const T*>(jb.B[k]), r, 1, A[k]);
  // X is streamed from global memory; each entry of X_hat is formed on the fly.
  const T* X = static_cast<const T*>(jb.X);
  const int nx = N[0] * N[1] * N[2];
  const double2 sx = fixed_sums2(nx, [&](int64_t e) {
    const int k = (int)(e % N[2]), j = (int)((e / N[2]) % N[1]), i = (int)(e / (N[1] * N[2]));
    T h = T(0);
    for (int q = 0; q < r; ++q) h = fma(A[0][i * r + q] * A[1][j * r + q], A[2][k * r + q], h);
    const double xv = (double)X[e], dv = xv - (double)h;
    return make_double2(dv * dv, xv * xv);
  }, red);
  if (threadIdx.x == 0) {
    nrm[0] = sx.x;
    nrm[1] = sx.y;
  }
  __syncthreads();
  if (threadIdx.x == 0 && rel_errs) rel_errs[blockIdx.x] = sqrt(nrm[0] / nrm[1]);
}

template <typename Job>
int upload(const Job* jobs, int n, Scratch& sc, Job** dev, cudaStream_t s) {
  NNC_TRY(sc.get(dev, (size_t)n));
  std::vector<Job> host(jobs, jobs + n);  // staged before cudaMemcpyAsync returns
  NNC_CUDA_TRY(cudaMemcpyAsync(*dev, host.data(), sizeof(Job) * n, cudaMemcpyHostToDevice, s));
  return NNC_OK;
}

}  // namespace

// Shared-memory elements of one two-pass nnCP job (see cpx_l2_kernel).
size_t cpx_l2_elems(const nncp_job& j) {
  const size_t N1 = j.m[0], N2 = j.m[1], N3 = j.m[2], r = j.r;
  const size_t t3 = N1 * N2 * r, t1 = r * N2 * N3;
  size_t nmax = N1 > N2 ? N1 : N2;
  nmax = nmax > N3 ? nmax : N3;
  return (N1 + N2 + N3) * r + 3 * r * r + (t3 > t1 ? t3 : t1) + 2 * nmax * r + r * r;
}

template <typename T>
int ntd_small_batched(int n_jobs, const ntd_small_job* jobs, int iters, double eps,
                      double* rel_errs, cudaStream_t s) {
  size_t elems = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const ntd_small_job& j = jobs[i];
    if (j.X == nullptr || j.G == nullptr) return NNC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
      if (j.dims[k] < 1 || j.m[k] < 1 || j.m[k] > 32 || j.F[k] == nullptr)
        return NNC_ERR_INVALID_ARG;
    const size_t e = ntd_small_elems(j);
    elems = e > elems ? e : elems;
  }
  const size_t smem = elems * sizeof(T);
  Scratch sc(s);
  ntd_small_job* dev = nullptr;
  long long work = 1;  // tuning class: largest tensor x largest multirank
  for (int i = 0; i < n_jobs; ++i) {
    long long w = 1;
    int mm = 1;
    for (int k = 0; k < 3; ++k) {
      w *= jobs[i].dims[k];
      mm = jobs[i].m[k] > mm ? jobs[i].m[k] : mm;
    }
    work = w * mm > work ? w * mm : work;
  }
  if (smem <= kSmemBudget) {
    NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
    NNC_CUDA_TRY(raise_smem_limit((const void*)ntd_small_kernel<T>, smem));
    const TuneKey key{kTuneNtdSmall, (int)sizeof(T), size_class(work), size_class(n_jobs)};
    return run_tuned(key, iters, kThreads, s, [&](int threads, int sweeps, bool last) -> int {
      ntd_small_kernel<T><<<n_jobs, threads, smem, s>>>(dev, sweeps, (T)eps,
                                                        last ? rel_errs : nullptr);
      note_launch(s);
      NNC_CUDA_TRY(cudaGetLastError());
      return NNC_OK;
    });
  }
  // Some X does not fit: the whole batch keeps X in global memory.
  size_t l2 = 0;
  int mmax = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const size_t e = ntd_l2_elems(jobs[i]);
    l2 = e > l2 ? e : l2;
    for (int k = 0; k < 3; ++k) mmax = jobs[i].m[k] > mmax ? jobs[i].m[k] : mmax;
  }
  const size_t smem2 = l2 * sizeof(T);
  if (smem2 > kSmemBudget || mmax > 16) {
    set_error_detail_text("batched nnTD: a job's pass results or multirank exceed one block");
    return NNC_ERR_UNSUPPORTED;
  }
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  const void* kern = mmax <= 8 ? (const void*)ntd_l2_kernel<T, 8> : (const void*)ntd_l2_kernel<T, 16>;
  NNC_CUDA_TRY(raise_smem_limit(kern, smem2));
  const TuneKey key{kTuneNtdL2, (int)sizeof(T), size_class(work), size_class(n_jobs)};
  return run_tuned(key, iters, kThreads, s, [&](int threads, int sweeps, bool last) -> int {
    double* out = last ? rel_errs : nullptr;
    if (mmax <= 8)
      ntd_l2_kernel<T, 8><<<n_jobs, threads, smem2, s>>>(dev, sweeps, (T)eps, out);
    else
      ntd_l2_kernel<T, 16><<<n_jobs, threads, smem2, s>>>(dev, sweeps, (T)eps, out);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  });
}

template <typename T>
int nncp_l2_batched(int n_jobs, const nncp_job* jobs, int iters, double eps, double* rel_errs,
                    int* statuses, cudaStream_t s) {
  size_t elems = 0;
  int rmax = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nncp_job& j = jobs[i];
    if (!nncp_job_valid(j)) continue;  // the kernel reports it in its status
    if (j.d != 3) {
      set_error_detail_text("batched nnCP: a 4-way job too large for shared memory");
      return NNC_ERR_UNSUPPORTED;
    }
    const size_t e = cpx_l2_elems(j);
    elems = e > elems ? e : elems;
    rmax = j.r > rmax ? j.r : rmax;
  }
  const size_t smem = elems * sizeof(T);
  if (smem > kSmemBudget || rmax > 16) {
    set_error_detail_text("batched nnCP: a job's pass results or rank exceed one block");
    return NNC_ERR_UNSUPPORTED;
  }
  Scratch sc(s);
  nncp_job* dev = nullptr;
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  const void* kern = rmax <= 8 ? (const void*)cpx_l2_kernel<T, 8> : (const void*)cpx_l2_kernel<T, 16>;
  NNC_CUDA_TRY(raise_smem_limit(kern, smem));
  long long work = 1;
  for (int i = 0; i < n_jobs; ++i) {
    if (!nncp_job_valid(jobs[i])) continue;
    const long long w = (long long)jobs[i].m[0] * jobs[i].m[1] * jobs[i].m[2] * jobs[i].r;
    work = w > work ? w : work;
  }
  const TuneKey key{kTuneCpxL2, (int)sizeof(T), size_class(work), size_class(n_jobs)};
  return run_tuned(key, iters, kThreads, s, [&](int threads, int sweeps, bool last) -> int {
    double* out = last ? rel_errs : nullptr;
    int* st = last ? statuses : nullptr;
    if (rmax <= 8)
      cpx_l2_kernel<T, 8><<<n_jobs, threads, smem, s>>>(dev, sweeps, (T)eps, out, st);
    else
      cpx_l2_kernel<T, 16><<<n_jobs, threads, smem, s>>>(dev, sweeps, (T)eps, out, st);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  });
}

template <typename T>
int nmf_small_batched(int n_jobs, const nmf_job* jobs, int iters, double eps, double* rel_errs,
                      cudaStream_t s) {
  size_t elems = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nmf_job& j = jobs[i];
    if (j.A == nullptr || j.F == nullptr || j.B == nullptr || j.N < 1 || j.r < 1 || j.m < 1)
      return NNC_ERR_INVALID_ARG;
    const size_t e = nmf_small_elems(j);
    elems = e > elems ? e : elems;
  }
  const size_t smem = elems * sizeof(T);
  if (smem > kSmemBudget) return NNC_ERR_UNSUPPORTED;
  Scratch sc(s);
  nmf_job* dev = nullptr;
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  NNC_CUDA_TRY(raise_smem_limit((const void*)nmf_small_kernel<T>, smem));
  long long work = 1;
  for (int i = 0; i < n_jobs; ++i) {
    const long long w = (long long)jobs[i].N * jobs[i].m * jobs[i].r;
    work = w > work ? w : work;
  }
  const TuneKey key{kTuneNmfSmall, (int)sizeof(T), size_class(work), size_class(n_jobs)};
  return run_tuned(key, iters, kThreads, s, [&](int threads, int sweeps, bool last) -> int {
    nmf_small_kernel<T><<<n_jobs, threads, smem, s>>>(dev, sweeps, (T)eps,
                                                      last ? rel_errs : nullptr);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  });
}

template <typename T>
int lifted_small_batched(int n_jobs, const lifted_job* jobs, double* rel_errs, cudaStream_t s) {
  size_t elems = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const lifted_job& j = jobs[i];
    if (j.X == nullptr || j.r < 1) return NNC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
      if (j.dims[k] < 1 || j.m[k] < 1 || j.F[k] == nullptr || j.B[k] == nullptr)
        return NNC_ERR_INVALID_ARG;
    const size_t e = lifted_small_elems(j);
    elems = e > elems ? e : elems;
  }
  const size_t smem = elems * sizeof(T);
  if (smem > kSmemBudget) return NNC_ERR_UNSUPPORTED;
  Scratch sc(s);
  lifted_job* dev = nullptr;
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  NNC_CUDA_TRY(raise_smem_limit((const void*)lifted_err_kernel<T>, smem));
  lifted_err_kernel<T><<<n_jobs, kThreads, smem, s>>>(dev, rel_errs);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

#define NNC_SMALL_INST(T)                                                                     \
  template int ntd_small_batched<T>(int, const ntd_small_job*, int, double, double*,         \
                                    cudaStream_t);                                          \
  template int nmf_small_batched<T>(int, const nmf_job*, int, double, double*, cudaStream_t); \
  template int lifted_small_batched<T>(int, const lifted_job*, double*, cudaStream_t);        \
  template int nncp_l2_batched<T>(int, const nncp_job*, int, double, double*, int*,         \
                                  cudaStream_t);
NNC_SMALL_INST(float)
NNC_SMALL_INST(double)
#undef NNC_SMALL_INST

}  // namespace nnc
