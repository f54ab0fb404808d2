// nnCPD of a 3-way core by one thread-block cluster per fit (Alg. 1, step 2):
// the Gauss-Seidel sweep of cpx_l2_kernel (small_batched.cu), a sweep
//   T   = G x_3 A3^T              MT1[i, q] = sum_j T[i, j, q] A2[j, q]    A1 <- MU
//                                 MT2[j, q] = sum_i T[i, j, q] A1[i, q]    A2 <- MU
//   T'  = G x_1 A1^T              MT3[k, q] = sum_j T'[q, j, k] A2[j, q]   A3 <- MU
// with A_n <- max(A_n * MT_n / max(A_n V_n, eps), 0), V_n the Hadamard product
// of the other factors' Grams, spread over kCl CTAs instead of one.
//
// CTA c of the cluster keeps, in shared memory, the slab of the core with
// i in [c ni, (c + 1) ni) (for T) and the slab with k in [c nk, (c + 1) nk)
// (for T'), and a copy of every factor and Gram. It forms T and T' on its
// slabs, MT1 and MT3 on its rows, and the new rows of A1 and A3 for its i and
// k; the MU step of A2 (whose MT2 sums over every i) runs in every CTA on the
// same data. Twice per sweep the CTAs exchange through distributed shared
// memory what the others need:
//   after A1:  its new A1 rows, its share of Gram1 and its share of MT2;
//   after A3:  its new A3 rows and its share of Gram3;
// each CTA writes them to an outbox of its own, the cluster synchronises, and
// every CTA reads all outboxes, adding the shares in CTA order (so every CTA
// holds bit-identical factors and Grams, and results do not depend on timing).
// The second exchange's barrier also tells every CTA that the first outbox has
// been read, and the next sweep's first barrier the same of the second, so two
// barriers per sweep suffice.
#include <cooperative_groups.h>

#include <vector>

#include "kernels.cuh"
#include "nncp.cuh"

namespace nnc {
namespace cg = cooperative_groups;
namespace {

constexpr int kCl = 8;  // CTAs per fit (the portable cluster size)
constexpr int kClThreads = 512;

__host__ __device__ constexpr size_t al4(size_t x) { return (x + 3) & ~static_cast<size_t>(3); }

// Element offsets of one CTA's shared memory.
struct ClLayout {
  int ni, nk;  // slab widths
  int xpitch;  // row pitch of the i-slab
  size_t xi, xk, a[3], g[3], tb, mt, den, v, ob1, ob2, total;
  __host__ __device__ explicit ClLayout(const int* N, int r) {
    ni = (N[0] + kCl - 1) / kCl;
    nk = (N[2] + kCl - 1) / kCl;
    int nmax = N[0] > N[1] ? N[0] : N[1];
    nmax = nmax > N[2] ? nmax : N[2];
    size_t p = 0;
    xpitch = N[2] | 1;  // odd: the rows a warp reads fall on distinct banks
    xi = p;  p += al4((size_t)ni * N[1] * xpitch);  // [ii][j][k], rows xpitch apart
    xk = p;  p += al4((size_t)N[0] * N[1] * nk);  // [i][j][kk]
    for (int n = 0; n < 3; ++n) { a[n] = p;  p += al4((size_t)N[n] * r); }
    for (int n = 0; n < 3; ++n) { g[n] = p;  p += al4((size_t)r * r); }
    const size_t t3 = (size_t)ni * N[1] * r, t1 = (size_t)N[1] * nk * r;
    tb = p;  p += al4(t3 > t1 ? t3 : t1);           // T [ii][j][q], then T' [j][kk][q]
    mt = p;  p += al4((size_t)nmax * r);
    den = p; p += al4((size_t)nmax * r);
    v = p;   p += al4((size_t)r * r);
    ob1 = p; p += al4((size_t)ni * r + (size_t)r * r + (size_t)N[1] * r);
    ob2 = p; p += al4((size_t)nk * r + (size_t)r * r);
    total = p;
  }
};

// out[e] = sum_{t < len} term(e, t, .) for e < nout, with term(e, t, s) =
// fma(x_t, y_t, s): for len >= 16 four consecutive lanes share an output,
// lane u adds the terms t = u, u + 4, ... in order, and a fixed shuffle tree
// adds the four partial sums (the reductions of the sweep are latency-bound;
// this keeps four times more of them in flight); shorter ones take one lane
// each, terms in order. Every thread of the block calls it.
template <typename T, typename F>
__device__ __forceinline__ void dots4(int nout, int len, F term, T* out) {
  if (len < 16) {  // too short to share: one lane per output
    for (int e = threadIdx.x; e < nout; e += blockDim.x) {
      T s = T(0);
      for (int t = 0; t < len; ++t) s = term(e, t, s);
      out[e] = s;
    }
    return;
  }
  const int per = blockDim.x / 4, u = threadIdx.x & 3;
  for (int e0 = 0; e0 < nout; e0 += per) {
    const int e = e0 + (int)threadIdx.x / 4;
    T s = T(0);
    if (e < nout)
      for (int t = u; t < len; t += 4) s = term(e, t, s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (e < nout && u == 0) out[e] = s;
  }
}

// gram[a, b] = sum_{i < n} A[i, a] A[i, b] (A: n x r, row-major).
template <typename T>
__device__ void gram_rows(const T* A, int n, int r, T* gram) {
  dots4<T>(r * r, n, [&](int e, int i, T s) {
    const int a = e / r, b = e - a * r;
    return fma(A[i * r + a], A[i * r + b], s);
  }, gram);
}

// MU on rows [0, n) of A (row-major, r wide) with numerators MT (n x r):
// A <- max(A * MT / max(A V, eps), 0). den is scratch, n x r.
template <typename T>
__device__ void mu_rows_local(T* A, const T* MT, const T* V, int n, int r, T eps, T* den) {
  dots4<T>(n * r, r, [&](int e, int p, T s) {
    const int i = e / r, q = e - i * r;
    return fma(A[i * r + p], V[p * r + q], s);
  }, den);
  __syncthreads();
  for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
    const T v = A[e] * MT[e] / (den[e] > eps ? den[e] : eps);
    A[e] = v > T(0) ? v : T(0);
  }
  __syncthreads();
}

// P[row, q] = sum_{t < len} x[row, t] F[t, q] for row < nrow, q < r, where
// x[row, t] = X[xo(row) + t xs] and F is len x r: four q per thread (four
// independent accumulators, F read in 16-byte rows) when r % 4 == 0.
template <typename T, typename XO>
__device__ void pass_quads(int nrow, int len, int r, const T* X, XO xo, int64_t xs, const T* F,
                           T* P) {
  if ((r & 3) == 0) {
    const int nq = r / 4;
    for (int e = threadIdx.x; e < nrow * nq; e += blockDim.x) {
      const int row = e / nq, q = 4 * (e - row * nq);
      const T* x = X + xo(row);
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll 4
      for (int t = 0; t < len; ++t) {
        const T v = x[t * xs];
        T f[4];
        if constexpr (sizeof(T) == 4) {  // F rows start on 16 bytes (r % 4 == 0)
          const float4 w = *reinterpret_cast<const float4*>(F + t * r + q);
          f[0] = w.x; f[1] = w.y; f[2] = w.z; f[3] = w.w;
        } else {
          const double2 w0 = *reinterpret_cast<const double2*>(F + t * r + q);
          const double2 w1 = *reinterpret_cast<const double2*>(F + t * r + q + 2);
          f[0] = w0.x; f[1] = w0.y; f[2] = w1.x; f[3] = w1.y;
        }
        a0 = fma(v, f[0], a0);
        a1 = fma(v, f[1], a1);
        a2 = fma(v, f[2], a2);
        a3 = fma(v, f[3], a3);
      }
      T* o = P + (size_t)row * r + q;
      o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3;
    }
  } else {
    dots4<T>(nrow * r, len, [&](int e, int t, T s) {
      const int row = e / r, q = e - row * r;
      return fma(X[xo(row) + t * xs], F[t * r + q], s);
    }, P);
  }
}

template <typename T>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads)
    cpx_cluster_kernel(const nncp_job* __restrict__ jobs, int iters, T eps, double* rel_errs,
                       int* statuses) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kFixedLanes];
  __shared__ double sums[2];
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int job = blockIdx.x / kCl;
  const nncp_job& jb = jobs[job];
  // A job the host skipped: every CTA of the cluster leaves before any
  // cluster barrier.
  if (!nncp_job_valid(jb) || jb.d != 3) {
    if (statuses != nullptr && c == 0 && threadIdx.x == 0) statuses[job] = NNC_ERR_INVALID_ARG;
    return;
  }
  const int N1 = jb.m[0], N2 = jb.m[1], N3 = jb.m[2], r = jb.r;
  const ClLayout L(jb.m, r);
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* Xi = sm + L.xi;
  T* Xk = sm + L.xk;
  T* A[3] = {sm + L.a[0], sm + L.a[1], sm + L.a[2]};
  T* Gr[3] = {sm + L.g[0], sm + L.g[1], sm + L.g[2]};
  T* Tb = sm + L.tb;
  T* MT = sm + L.mt;
  T* den = sm + L.den;
  T* V = sm + L.v;
  T* ob1 = sm + L.ob1;  // [A1 rows: ni x r][Gram1 share: r x r][MT2 share: N2 x r]
  T* ob2 = sm + L.ob2;  // [A3 rows: nk x r][Gram3 share: r x r]
  const int i0 = c * L.ni, ni = max(0, min(L.ni, N1 - i0));
  const int k0 = c * L.nk, nk = max(0, min(L.nk, N3 - k0));
  const T* X = static_cast<const T*>(jb.G);
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < ni * N2 * N3; e += nt) {
    const int row = e / N3, k = e - row * N3;
    Xi[row * L.xpitch + k] = X[(int64_t)i0 * N2 * N3 + e];
  }
  for (int e = tid; e < N1 * N2 * nk; e += nt) {
    const int kk = e % nk, ij = e / nk;
    Xk[e] = X[(int64_t)ij * N3 + k0 + kk];
  }
  for (int n = 0; n < 3; ++n) {
    const T* src = static_cast<const T*>(jb.B[n]);
    for (int e = tid; e < jb.m[n] * r; e += nt) A[n][e] = src[e];
  }
  __syncthreads();
  for (int n = 0; n < 3; ++n) gram_rows(A[n], jb.m[n], r, Gr[n]);
  __syncthreads();

  for (int it = 0; it < iters; ++it) {
    // ---- T[ii, j, q] = sum_k Xi[ii, j, k] A3[k, q]; MT1 on this CTA's rows --
    pass_quads<T>(ni * N2, N3, r, Xi, [&](int row) { return (int64_t)row * L.xpitch; }, 1, A[2],
                  Tb);
    for (int e = tid; e < r * r; e += nt) V[e] = Gr[1][e] * Gr[2][e];
    __syncthreads();
    dots4<T>(ni * r, N2, [&](int e, int j, T s) {
      const int ii = e / r, q = e - ii * r;
      return fma(Tb[(ii * N2 + j) * r + q], A[1][j * r + q], s);
    }, MT);
    __syncthreads();
    // ---- the new rows i0 .. i0 + ni - 1 of A1 ---------------------------------
    mu_rows_local(A[0] + (size_t)i0 * r, MT, V, ni, r, eps, den);
    // ---- outbox 1: those rows, their Gram share, their MT2 share --------------
    {
      const T* a1 = A[0] + (size_t)i0 * r;
      for (int e = tid; e < ni * r; e += nt) ob1[e] = a1[e];
      gram_rows(a1, ni, r, ob1 + L.ni * r);
      dots4<T>(N2 * r, ni, [&](int e, int ii, T s) {
        const int j = e / r, q = e - j * r;
        return fma(Tb[(ii * N2 + j) * r + q], a1[ii * r + q], s);
      }, ob1 + L.ni * r + r * r);
    }
    cl.sync();
    // ---- gather A1, Gram1 and MT2 from every CTA, shares added in CTA order ---
    for (int e = tid; e < r * r + N2 * r; e += nt) {
      T v[kCl];
#pragma unroll
      for (int c2 = 0; c2 < kCl; ++c2) v[c2] = cl.map_shared_rank(ob1, c2)[L.ni * r + e];
      T acc = v[0];
#pragma unroll
      for (int c2 = 1; c2 < kCl; ++c2) acc += v[c2];
      if (e < r * r) Gr[0][e] = acc;
      else MT[e - r * r] = acc;
    }
    for (int e = tid; e < N1 * r; e += nt) {
      const int c2 = (e / r) / L.ni;
      A[0][e] = cl.map_shared_rank(ob1, c2)[e - c2 * L.ni * r];
    }
    __syncthreads();
    // ---- A2 in every CTA alike -------------------------------------------------
    for (int e = tid; e < r * r; e += nt) V[e] = Gr[0][e] * Gr[2][e];
    __syncthreads();
    mu_rows_local(A[1], MT, V, N2, r, eps, den);
    // ---- T'[j, kk, q] = sum_i A1[i, q] Xk[i, j, kk]; MT3 on this CTA's rows ---
    gram_rows(A[1], N2, r, Gr[1]);
    pass_quads<T>(N2 * nk, N1, r, Xk, [&](int jk) { return (int64_t)jk; }, (int64_t)N2 * nk,
                  A[0], Tb);
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) V[e] = Gr[0][e] * Gr[1][e];
    dots4<T>(nk * r, N2, [&](int e, int j, T s) {
      const int kk = e / r, q = e - kk * r;
      return fma(Tb[(j * nk + kk) * r + q], A[1][j * r + q], s);
    }, MT);
    __syncthreads();
    // ---- the new rows k0 .. k0 + nk - 1 of A3; outbox 2 -----------------------
    mu_rows_local(A[2] + (size_t)k0 * r, MT, V, nk, r, eps, den);
    {
      const T* a3 = A[2] + (size_t)k0 * r;
      for (int e = tid; e < nk * r; e += nt) ob2[e] = a3[e];
      gram_rows(a3, nk, r, ob2 + L.nk * r);
    }
    cl.sync();
    for (int e = tid; e < r * r; e += nt) {
      T v[kCl];
#pragma unroll
      for (int c2 = 0; c2 < kCl; ++c2) v[c2] = cl.map_shared_rank(ob2, c2)[L.nk * r + e];
      T acc = v[0];
#pragma unroll
      for (int c2 = 1; c2 < kCl; ++c2) acc += v[c2];
      Gr[2][e] = acc;
    }
    for (int e = tid; e < N3 * r; e += nt) {
      const int c2 = (e / r) / L.nk;
      A[2][e] = cl.map_shared_rank(ob2, c2)[e - c2 * L.nk * r];
    }
    __syncthreads();
  }

  // ||G - I x_k A_k||^2 and ||G||^2 on this CTA's slab (FP64, in an order fixed
  // by the slab alone), then added over the cluster in CTA order.
  const double2 part = fixed_sums2((int64_t)ni * N2 * N3, [&](int64_t e) {
    const int k = (int)(e % N3), ij = (int)(e / N3), j = ij % N2, ii = ij / N2;
    T hat = T(0);
    for (int q = 0; q < r; ++q)
      hat = fma(A[0][(i0 + ii) * r + q] * A[1][j * r + q], A[2][k * r + q], hat);
    const double g = (double)Xi[ij * L.xpitch + k], d = g - (double)hat;
    return make_double2(d * d, g * g);
  }, red);
  if (tid == 0) {
    sums[0] = part.x;
    sums[1] = part.y;
  }
  cl.sync();
  if (c == 0) {
    bool finite = true;
    for (int n = 0; n < 3; ++n) {
      T* dst = static_cast<T*>(jb.B[n]);
      for (int e = tid; e < jb.m[n] * r; e += nt) {
        dst[e] = A[n][e];
        finite = finite && isfinite(A[n][e]);
      }
    }
    const int ok = __syncthreads_and(finite ? 1 : 0);
    if (tid == 0) {
      double d2 = 0.0, x2 = 0.0;
      for (int s = 0; s < kCl; ++s) {
        const double* o = cl.map_shared_rank(sums, s);
        d2 += o[0];
        x2 += o[1];
      }
      if (rel_errs) rel_errs[job] = x2 > 0.0 ? sqrt(d2 / x2) : sqrt(d2);
      if (statuses)
        statuses[job] = (ok && isfinite(d2) && isfinite(x2)) ? NNC_OK : NNC_ERR_NONFINITE;
    }
  }
  // No CTA leaves while another may still read its shared memory.
  cl.sync();
}

}  // namespace

size_t cpx_cluster_elems(const nncp_job& j) { return ClLayout(j.m, j.r).total; }

int cpx_cluster_ctas() { return kCl; }

template <typename T>
int nncp_cluster_batched(int n_jobs, const nncp_job* jobs, int iters, double eps,
                         double* rel_errs, int* statuses, cudaStream_t s) {
  size_t elems = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const nncp_job& j = jobs[i];
    if (!nncp_job_valid(j)) continue;  // the kernel reports it in its status
    if (j.d != 3) {
      set_error_detail_text("cluster nnCP: a 4-way job");
      return NNC_ERR_UNSUPPORTED;
    }
    const size_t e = cpx_cluster_elems(j);
    elems = e > elems ? e : elems;
  }
  const size_t smem = elems * sizeof(T);
  if (smem > kSmemBudget) {
    set_error_detail_text("cluster nnCP: a job's slabs exceed one block of shared memory");
    return NNC_ERR_UNSUPPORTED;
  }
  Scratch sc(s);
  nncp_job* dev = nullptr;
  NNC_TRY(sc.get(&dev, (size_t)n_jobs));
  std::vector<nncp_job> host(jobs, jobs + n_jobs);  // staged before cudaMemcpyAsync returns
  NNC_CUDA_TRY(cudaMemcpyAsync(dev, host.data(), sizeof(nncp_job) * n_jobs,
                               cudaMemcpyHostToDevice, s));
  NNC_CUDA_TRY(raise_smem_limit((const void*)cpx_cluster_kernel<T>, smem));
  cpx_cluster_kernel<T><<<(unsigned)(n_jobs * kCl), kClThreads, smem, s>>>(dev, iters, (T)eps,
                                                                           rel_errs, statuses);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template int nncp_cluster_batched<float>(int, const nncp_job*, int, double, double*, int*,
                                         cudaStream_t);
template int nncp_cluster_batched<double>(int, const nncp_job*, int, double, double*, int*,
                                          cudaStream_t);

}  // namespace nnc
