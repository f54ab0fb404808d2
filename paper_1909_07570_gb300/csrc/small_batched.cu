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

#include "small_batched.cuh"

namespace nnc {
namespace {

constexpr int kThreads = 256;

// out = in x_k A for a 3-way `in` (dims d[0..2], C order): out has d[k]
// replaced by P and out[.., p, ..] = sum_j A[p sp + j sj] in[.., j, ..].
template <typename T>
__device__ void mp3(const T* in, const int* d, int k, const T* A, int sp, int sj, int P, T* out) {
  int od[3] = {d[0], d[1], d[2]};
  od[k] = P;
  const int n = od[0] * od[1] * od[2];
  const int J = d[k];
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int idx[3];
    idx[2] = e % od[2];
    idx[1] = (e / od[2]) % od[1];
    idx[0] = e / (od[1] * od[2]);
    const int p = idx[k];
    T s = T(0);
    for (int j = 0; j < J; ++j) {
      idx[k] = j;
      s = fma(A[p * sp + j * sj], in[(idx[0] * d[1] + idx[1]) * d[2] + idx[2]], s);
    }
    out[e] = s;
  }
  __syncthreads();
}

// out[i, a] = sum over the other two indices of Y[.., i, ..] G[.., a, ..]
// (unfold_n(Y) unfold_n(G)^T); Y has dims dy, G has dims dg, equal off mode n.
template <typename T>
__device__ void unfold_dot(const T* Y, const int* dy, const T* G, const int* dg, int n, T* out) {
  const int NI = dy[n], MA = dg[n];
  const int o0 = n == 0 ? 1 : 0, o1 = n == 2 ? 1 : 2;
  for (int e = threadIdx.x; e < NI * MA; e += blockDim.x) {
    const int i = e / MA, a = e % MA;
    T s = T(0);
    for (int u = 0; u < dy[o0]; ++u)
      for (int v = 0; v < dy[o1]; ++v) {
        int iy[3], ig[3];
        iy[n] = i;
        ig[n] = a;
        iy[o0] = ig[o0] = u;
        iy[o1] = ig[o1] = v;
        s = fma(Y[(iy[0] * dy[1] + iy[1]) * dy[2] + iy[2]],
                G[(ig[0] * dg[1] + ig[1]) * dg[2] + ig[2]], s);
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

// sum (a - b)^2 and sum a^2 in FP64 over n entries (b may be null: 0).
template <typename T>
__device__ void diff_norms(const T* a, const T* b, int n, double* red, double* out2) {
  double s = 0.0, x = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const double av = (double)a[e], bv = b ? (double)b[e] : 0.0;
    s += (av - bv) * (av - bv);
    x += av * av;
  }
  s = block_sum(s, red);
  x = block_sum(x, red);
  if (threadIdx.x == 0) {
    out2[0] = s;
    out2[1] = x;
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
  __shared__ double red[32];
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

size_t nmf_small_elems(const nmf_job& j) {
  const size_t N = j.N, r = j.r, m = j.m;
  return N * r + N * m + m * r + 2 * m * m + 2 * N * m + 2 * m * r + N * r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
nmf_small_kernel(const nmf_job* __restrict__ jobs, int iters, T eps, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
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
  size_t a = 0, nx = 1;
  for (int k = 0; k < 3; ++k) {
    a += (size_t)j.dims[k] * j.r;
    nx *= j.dims[k];
  }
  return a + nx;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
lifted_err_kernel(const lifted_job* __restrict__ jobs, double* rel_errs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ double nrm[2];
  const lifted_job& jb = jobs[blockIdx.x];
  const int* N = jb.dims;
  const int r = jb.r;
  T* A[3];
  A[0] = reinterpret_cast<T*>(smem_raw);
  A[1] = A[0] + N[0] * r;
  A[2] = A[1] + N[1] * r;
  T* Xh = A[2] + N[2] * r;
  for (int k = 0; k < 3; ++k)  // A_k = F_k B_k
    sgemm(N[k], r, jb.m[k], static_cast<const T*>(jb.F[k]), jb.m[k], 1,
          static_cast<const T*>(jb.B[k]), r, 1, A[k]);
  const int nx = N[0] * N[1] * N[2];
  for (int e = threadIdx.x; e < nx; e += blockDim.x) {
    const int k = e % N[2], j = (e / N[2]) % N[1], i = e / (N[1] * N[2]);
    T s = T(0);
    for (int q = 0; q < r; ++q) s = fma(A[0][i * r + q] * A[1][j * r + q], A[2][k * r + q], s);
    Xh[e] = s;
  }
  __syncthreads();
  diff_norms(static_cast<const T*>(jb.X), Xh, nx, red, nrm);
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
  if (smem > 200 * 1024) return NNC_ERR_UNSUPPORTED;
  Scratch sc(s);
  ntd_small_job* dev = nullptr;
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  NNC_CUDA_TRY(raise_smem_limit((const void*)ntd_small_kernel<T>, smem));
  ntd_small_kernel<T><<<n_jobs, kThreads, smem, s>>>(dev, iters, (T)eps, rel_errs);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
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
  if (smem > 200 * 1024) return NNC_ERR_UNSUPPORTED;
  Scratch sc(s);
  nmf_job* dev = nullptr;
  NNC_TRY(upload(jobs, n_jobs, sc, &dev, s));
  NNC_CUDA_TRY(raise_smem_limit((const void*)nmf_small_kernel<T>, smem));
  nmf_small_kernel<T><<<n_jobs, kThreads, smem, s>>>(dev, iters, (T)eps, rel_errs);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
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
  if (smem > 200 * 1024) return NNC_ERR_UNSUPPORTED;
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
  template int lifted_small_batched<T>(int, const lifted_job*, double*, cudaStream_t);
NNC_SMALL_INST(float)
NNC_SMALL_INST(double)
#undef NNC_SMALL_INST

}  // namespace nnc
