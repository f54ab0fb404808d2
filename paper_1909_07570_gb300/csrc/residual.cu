// The lift A^(n) = F^(n) B^(n) and the one-pass reconstruction residual.
//
// recon_residual streams X once. The model is first reduced to rows U[t, :]
// (length K = m_d for Tucker, r for CP), t running over (i_1, ..., i_{d-1}):
//   Tucker: U = G x_1 F^(1) ... x_{d-1} F^(d-1)
//   CP:     U[t, q] = A^(1)[i_1, q] ... A^(d-1)[i_{d-1}, q]
// and X_hat[t, k] = sum_c U[t, c] F^(d)[k, c] (A^(d) for CP), by
// Eq. TD:matrix-format and Eq. CPD:matrix-format contracted mode by mode.
// The streaming kernel gives each thread one k (F^(d)[k, :] in registers) and
// a tile of rows (U rows in shared memory), forms X_hat in T and accumulates
// (x - x_hat)^2 and x^2 (FP32 per thread for float data, FP64 across threads
// and blocks); per-block partials are added in block order.
#include "kernels.cuh"
#include "residual.cuh"

namespace nnc {
namespace {

template <typename T>
__global__ void lift_kernel(const T* __restrict__ F, const T* __restrict__ B, int64_t N, int M,
                            int r, T* __restrict__ A) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int q = (int)(e % r);
    T s = T(0);
    for (int a = 0; a < M; ++a) s = fma(F[i * M + a], B[(int64_t)a * r + q], s);
    A[e] = s;
  }
}

// out[l, q, c] = sum_j A[q, j] Y[l, j, c] for any Q (one thread per output).
template <typename T>
__global__ void mode_product_any_kernel(const T* __restrict__ Y, int64_t L, int J, int64_t C,
                                        const T* __restrict__ A, int Q, T* __restrict__ out) {
  const int64_t n = L * Q * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % C;
    const int64_t q = (e / C) % Q;
    const int64_t l = e / (C * Q);
    const T* y = Y + l * J * C + c;
    const T* a = A + q * J;
    T s = T(0);
    for (int j = 0; j < J; ++j) s = fma(a[j], y[(int64_t)j * C], s);
    out[e] = s;
  }
}

template <typename T>
__global__ void cp_rows_kernel(const T* __restrict__ A1, const T* __restrict__ A2, int64_t N1,
                               int64_t N2, int r, T* __restrict__ U) {
  const int64_t n = N1 * N2 * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % r);
    const int64_t j = (e / r) % N2;
    const int64_t i = e / (r * N2);
    U[e] = A1[i * r + q] * A2[j * r + q];
  }
}

constexpr int kResThreads = 256;
constexpr int kResRows = 64;

// Block (k tile of kResThreads, row tile of kResRows). Thread k keeps F3[k, :]
// in registers (KM >= K entries, zero past K); the block's U rows sit in
// shared memory and are read as broadcasts. Per element: x_hat = U[t, :] .
// F3[k, :] in T, then (x - x_hat)^2 and x^2. For T = float the thread adds its
// rows' terms in FP32 (rounded to nearest, so the errors are unbiased and
// shrink in the FP64 sums that follow); GB300's FP64 rate is far below its
// FP32 rate, and FP64 arithmetic per element would bound the pass. The block
// sums and the partials are FP64.
template <typename T, int KM>
__global__ void __launch_bounds__(kResThreads)
residual_stream_kernel(const T* __restrict__ X, int64_t R, int64_t N3, const T* __restrict__ U,
                       int K, const T* __restrict__ F3, double* __restrict__ part) {
  __shared__ __align__(16) T us[kResRows * KM];
  __shared__ double red[32];
  const int64_t k = (int64_t)blockIdx.x * kResThreads + threadIdx.x;
  const bool act = k < N3;
  T f[KM];
#pragma unroll
  for (int c = 0; c < KM; ++c) f[c] = (act && c < K) ? F3[k * K + c] : T(0);
  const int64_t r0 = (int64_t)blockIdx.y * kResRows;
  const int nr = (int)(r0 + kResRows < R ? kResRows : R - r0);
  for (int e = threadIdx.x; e < nr * KM; e += kResThreads) {
    const int row = e / KM, c = e % KM;
    us[e] = c < K ? U[(r0 + row) * K + c] : T(0);
  }
  __syncthreads();
  T d2 = T(0), x2 = T(0);
  if (act) {
    const T* xp = X + r0 * N3 + k;
#pragma unroll 4
    for (int row = 0; row < nr; ++row) {
      const T x = xp[(int64_t)row * N3];
      const T* u = us + row * KM;
      T h0 = T(0), h1 = T(0);
#pragma unroll
      for (int c = 0; c < KM; c += 2) {
        h0 = fma(u[c], f[c], h0);
        h1 = fma(u[c + 1], f[c + 1], h1);
      }
      const T dd = x - (h0 + h1);
      d2 = fma(dd, dd, d2);
      x2 = fma(x, x, x2);
    }
  }
  double td2 = (double)d2, tx2 = (double)x2;
  if (act && !(isfinite(d2) && isfinite(x2))) {
    // The FP32 terms overflowed (entries beyond about 1e19): these rows again
    // with FP64 terms. Non-finite data stays non-finite.
    td2 = 0.0;
    tx2 = 0.0;
    const T* xp = X + r0 * N3 + k;
    for (int row = 0; row < nr; ++row) {
      const double x = (double)xp[(int64_t)row * N3];
      double h = 0.0;
      for (int c = 0; c < KM; ++c) h = fma((double)us[row * KM + c], (double)f[c], h);
      const double dd = x - h;
      td2 += dd * dd;
      tx2 += x * x;
    }
  }
  const double bd2 = block_sum(td2, red);
  const double bx2 = block_sum(tx2, red);
  if (threadIdx.x == 0) {
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * b] = bd2;
    part[2 * b + 1] = bx2;
  }
}

// The block partials added in block order; out (2 doubles) and/or rel_out
// (sqrt(d2 / x2), e.g. a trace slot) may be NULL.
__global__ void residual_final_kernel(const double* __restrict__ part, int64_t nblocks,
                                      double* out, double* rel_out) {
  __shared__ double red[32];
  double d2 = 0.0, x2 = 0.0;
  for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) {
    d2 += part[2 * b];
    x2 += part[2 * b + 1];
  }
  d2 = block_sum(d2, red);
  x2 = block_sum(x2, red);
  if (threadIdx.x == 0) {
    if (out) {
      out[0] = d2;
      out[1] = x2;
    }
    if (rel_out) *rel_out = sqrt(d2 / x2);
  }
}

unsigned grid_cap(int64_t n, int threads) {
  int64_t b = ceil_div(n, threads);
  if (b > 8192) b = 8192;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t launch_lift(const T* F, const T* B, int64_t N, int M, int r, T* A, cudaStream_t s) {
  lift_kernel<T><<<grid_cap(N * r, 256), 256, 0, s>>>(F, B, N, M, r, A);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T>
int residual_prepare(int d, const int64_t* dims, int model, const int* m, int r, Scratch& sc,
                     ResidualWork<T>* w) {
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  *w = ResidualWork<T>{};
  const int K = model == 0 ? m[d - 1] : r;
  int64_t R = 1;  // rows of U: N_1 ... N_{d-1}
  for (int k = 0; k < d - 1; ++k) R *= dims[k];
  NNC_TRY(sc.get(&w->U, (size_t)(R * K)));
  if (model == 0) {
    int64_t lead = 1, tail = 1;
    for (int k = 1; k < d; ++k) tail *= m[k];
    for (int k = 0; k < d - 2; ++k) {
      const int64_t n_out = lead * dims[k] * (tail);
      NNC_TRY(sc.get(&w->tmp[k & 1], (size_t)n_out));
      lead *= dims[k];
      tail /= m[k + 1];
    }
  } else {
    int64_t rows = dims[0];
    for (int k = 1; k < d - 2; ++k) {
      NNC_TRY(sc.get(&w->tmp[0], (size_t)(rows * dims[k] * r)));
      rows *= dims[k];
    }
  }
  const int64_t Nd = dims[d - 1];
  w->nblocks = ceil_div(Nd, kResThreads) * ceil_div(R, kResRows);
  NNC_TRY(sc.get(&w->part, (size_t)(2 * w->nblocks)));
  return NNC_OK;
}

template <typename T>
int residual_run(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                 const T* const* factors, const T* G, const ResidualWork<T>& w, double* out2,
                 double* rel_out, cudaStream_t s) {
  const int K = model == 0 ? m[d - 1] : r;
  int64_t R = 1;
  for (int k = 0; k < d - 1; ++k) R *= dims[k];
  T* U = w.U;
  if (model == 0) {
    // Mode products of the core with F^(1) .. F^(d-1), the last one into U:
    // cur[t_<k, i_k, c_>k] = sum_a F^(k)[i_k, a] prev[t_<k, a, c_>k].
    int64_t lead = 1;  // N_1 ... N_{k-1}
    int64_t tail = 1;  // m_{k+1} ... m_d
    for (int k = 1; k < d; ++k) tail *= m[k];
    const T* src = G;
    for (int k = 0; k < d - 1; ++k) {
      const int64_t n_out = lead * dims[k] * tail;
      T* dst = k < d - 2 ? w.tmp[k & 1] : U;
      mode_product_any_kernel<T><<<grid_cap(n_out, 256), 256, 0, s>>>(
          src, lead, m[k], tail, factors[k], (int)dims[k], dst);
      note_launch(s);
      src = dst;
      lead *= dims[k];
      tail /= m[k + 1];
    }
  } else {
    // U_k = U_{k-1} (.) A^(k) row by row: (rows of U_{k-1}) x N_k rows.
    int64_t rows = dims[0];
    const T* src = factors[0];
    for (int k = 1; k < d - 1; ++k) {
      T* dst = k < d - 2 ? w.tmp[0] : U;
      cp_rows_kernel<T><<<grid_cap(rows * dims[k] * r, 256), 256, 0, s>>>(src, factors[k], rows,
                                                                           dims[k], r, dst);
      note_launch(s);
      src = dst;
      rows *= dims[k];
    }
  }
  NNC_CUDA_TRY(cudaGetLastError());
  const T* Fd = factors[d - 1];  // F^(d) (Tucker) or A^(d) (CP): N_d x K
  const int64_t Nd = dims[d - 1];
  dim3 grid((unsigned)ceil_div(Nd, kResThreads), (unsigned)ceil_div(R, kResRows));
  if (K <= 16)
    residual_stream_kernel<T, 16><<<grid, kResThreads, 0, s>>>(X, R, Nd, U, K, Fd, w.part);
  else if (K <= 32)
    residual_stream_kernel<T, 32><<<grid, kResThreads, 0, s>>>(X, R, Nd, U, K, Fd, w.part);
  else if (K <= 64)
    residual_stream_kernel<T, 64><<<grid, kResThreads, 0, s>>>(X, R, Nd, U, K, Fd, w.part);
  else
    return NNC_ERR_UNSUPPORTED;
  note_launch(s);
  residual_final_kernel<<<1, 1024, 0, s>>>(w.part, w.nblocks, out2, rel_out);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int residual_device(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                    const T* const* factors, const T* G, double* out2, Scratch& sc,
                    cudaStream_t s) {
  ResidualWork<T> w;
  NNC_TRY(residual_prepare<T>(d, dims, model, m, r, sc, &w));
  return residual_run<T>(X, d, dims, model, m, r, factors, G, w, out2, nullptr, s);
}

template cudaError_t launch_lift<float>(const float*, const float*, int64_t, int, int, float*,
                                        cudaStream_t);
template cudaError_t launch_lift<double>(const double*, const double*, int64_t, int, int, double*,
                                         cudaStream_t);
template int residual_prepare<float>(int, const int64_t*, int, const int*, int, Scratch&,
                                     ResidualWork<float>*);
template int residual_prepare<double>(int, const int64_t*, int, const int*, int, Scratch&,
                                      ResidualWork<double>*);
template int residual_run<float>(const float*, int, const int64_t*, int, const int*, int,
                                 const float* const*, const float*, const ResidualWork<float>&,
                                 double*, double*, cudaStream_t);
template int residual_run<double>(const double*, int, const int64_t*, int, const int*, int,
                                  const double* const*, const double*,
                                  const ResidualWork<double>&, double*, double*, cudaStream_t);
template int residual_device<float>(const float*, int, const int64_t*, int, const int*, int,
                                    const float* const*, const float*, double*, Scratch&,
                                    cudaStream_t);
template int residual_device<double>(const double*, int, const int64_t*, int, const int*, int,
                                     const double* const*, const double*, double*, Scratch&,
                                     cudaStream_t);

}  // namespace nnc
