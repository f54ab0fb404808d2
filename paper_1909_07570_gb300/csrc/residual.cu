// The lift A^(n) = F^(n) B^(n) and the one-pass reconstruction residual.
//
// recon_residual streams X once. The model is first reduced to rows U[t, :]
// (length K = m_d for Tucker, r for CP), t running over (i_1, ..., i_{d-1}):
//   Tucker: U = G x_1 F^(1) ... x_{d-1} F^(d-1)
//   CP:     U[t, q] = A^(1)[i_1, q] ... A^(d-1)[i_{d-1}, q]
// and X_hat[t, k] = sum_c U[t, c] F^(d)[k, c] (A^(d) for CP), by
// Eq. TD:matrix-format and Eq. CPD:matrix-format contracted mode by mode.
// The streaming kernel holds the last factor transposed in shared memory,
// gives each thread one k of a row, forms X_hat in T and accumulates
// (x - x_hat)^2 and x^2 in FP64; per-block partials are added in block order.
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

template <typename T>
__global__ void __launch_bounds__(kResThreads)
residual_stream_kernel(const T* __restrict__ X, int64_t R, int64_t N3, const T* __restrict__ U,
                       int K, const T* __restrict__ F3, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ft = reinterpret_cast<T*>(smem_raw);  // K x kResThreads, transposed chunk of F3
  __shared__ double red[32];
  const int64_t k = (int64_t)blockIdx.x * kResThreads + threadIdx.x;
  const bool act = k < N3;
  for (int c = 0; c < K; ++c) ft[c * kResThreads + threadIdx.x] = act ? F3[k * K + c] : T(0);
  __syncthreads();
  double d2 = 0.0, x2 = 0.0;
  const int64_t r0 = (int64_t)blockIdx.y * kResRows;
  const int64_t r1 = r0 + kResRows < R ? r0 + kResRows : R;
  if (act) {
    for (int64_t row = r0; row < r1; ++row) {
      const T* u = U + row * K;
      T hat = T(0);
      for (int c = 0; c < K; ++c) hat = fma(u[c], ft[c * kResThreads + threadIdx.x], hat);
      const double x = (double)X[row * N3 + k];
      const double dd = x - (double)hat;
      d2 += dd * dd;
      x2 += x * x;
    }
  }
  d2 = block_sum(d2, red);
  x2 = block_sum(x2, red);
  if (threadIdx.x == 0) {
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * b] = d2;
    part[2 * b + 1] = x2;
  }
}

__global__ void residual_final_kernel(const double* __restrict__ part, int64_t nblocks,
                                      double* out) {
  __shared__ double red[32];
  double d2 = 0.0, x2 = 0.0;
  for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) {
    d2 += part[2 * b];
    x2 += part[2 * b + 1];
  }
  d2 = block_sum(d2, red);
  x2 = block_sum(x2, red);
  if (threadIdx.x == 0) {
    out[0] = d2;
    out[1] = x2;
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
int residual_device(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                    const T* const* factors, const T* G, double* out2, Scratch& sc,
                    cudaStream_t s) {
  if (d != 3 && d != 4) return NNC_ERR_INVALID_ARG;
  const int K = model == 0 ? m[d - 1] : r;
  int64_t R = 1;  // rows of U: N_1 ... N_{d-1}
  for (int k = 0; k < d - 1; ++k) R *= dims[k];
  T* U = nullptr;
  NNC_TRY(sc.get(&U, (size_t)(R * K)));
  if (model == 0) {
    // Mode products of the core with F^(1) .. F^(d-1), the last one into U:
    // cur[t_<k, i_k, c_>k] = sum_a F^(k)[i_k, a] prev[t_<k, a, c_>k].
    int64_t lead = 1;  // N_1 ... N_{k-1}
    int64_t tail = 1;  // m_{k+1} ... m_d
    for (int k = 1; k < d; ++k) tail *= m[k];
    const T* src = G;
    T* bufs[2] = {nullptr, nullptr};
    for (int k = 0; k < d - 1; ++k) {
      const int64_t n_out = lead * dims[k] * tail;
      T* dst = U;
      if (k < d - 2) {
        if (!bufs[k & 1]) NNC_TRY(sc.get(&bufs[k & 1], (size_t)n_out));
        dst = bufs[k & 1];
      }
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
    T* tmp = nullptr;
    for (int k = 1; k < d - 1; ++k) {
      T* dst = U;
      if (k < d - 2) {
        NNC_TRY(sc.get(&tmp, (size_t)(rows * dims[k] * r)));
        dst = tmp;
      }
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
  const int64_t nblocks = (int64_t)grid.x * grid.y;
  double* part = nullptr;
  NNC_TRY(sc.get(&part, (size_t)(2 * nblocks)));
  const size_t smem = (size_t)K * kResThreads * sizeof(T);
  if (smem > 48 * 1024)
    NNC_CUDA_TRY(raise_smem_limit((const void*)residual_stream_kernel<T>, smem));
  residual_stream_kernel<T><<<grid, kResThreads, smem, s>>>(X, R, Nd, U, K, Fd, part);
  note_launch(s);
  residual_final_kernel<<<1, 1024, 0, s>>>(part, nblocks, out2);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template cudaError_t launch_lift<float>(const float*, const float*, int64_t, int, int, float*,
                                        cudaStream_t);
template cudaError_t launch_lift<double>(const double*, const double*, int64_t, int, int, double*,
                                         cudaStream_t);
template int residual_device<float>(const float*, int, const int64_t*, int, const int*, int,
                                    const float* const*, const float*, double*, Scratch&,
                                    cudaStream_t);
template int residual_device<double>(const double*, int, const int64_t*, int, const int*, int,
                                     const double* const*, const double*, double*, Scratch&,
                                     cudaStream_t);

}  // namespace nnc
