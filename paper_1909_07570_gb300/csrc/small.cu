// Core-sized and factor-sized kernels of an nnTD sweep: unfolding products
// (numerators Num_n and the m_n x m_n matrices of the denominators), the
// multiplicative updates with their nonnegativity projection, the FP64
// residual identity and the one-pass statistics of X.
#include "kernels.cuh"

namespace nnc {
namespace {

// One block per output row i: the slice Y[:, i, :] is staged in shared memory,
// then each warp takes outputs a = warp, warp + nwarps, ... and sums
// Y[l, i, c] * G[l, a, c] over the flattened (l, c) with its lanes.
template <typename T>
__global__ void pair_contract_kernel(const T* __restrict__ Y, const T* __restrict__ G, int64_t L,
                                     int NI, int MA, int64_t C, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);
  const int i = blockIdx.x;
  const int64_t LC = L * C;
  for (int64_t e = threadIdx.x; e < LC; e += blockDim.x) {
    const int64_t l = e / C, c = e % C;
    ys[e] = Y[(l * NI + i) * C + c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int a = warp; a < MA; a += nwarps) {
    T s = T(0);
    for (int64_t e = lane; e < LC; e += 32) {
      const int64_t l = e / C, c = e % C;
      s = fma(ys[e], G[(l * MA + a) * C + c], s);
    }
    s = warp_sum(s);
    if (lane == 0) out[(int64_t)i * MA + a] = s;
  }
}

// Rows of F are updated by one group of M' = roundup(M, 32) threads each; the
// old row is staged in shared memory before any entry of it is overwritten.
template <typename T>
__global__ void factor_mu_kernel(T* __restrict__ F, const T* __restrict__ Num,
                                 const T* __restrict__ H, int64_t N, int M, int MP, T eps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* hs = reinterpret_cast<T*>(smem_raw);  // M x M
  T* fs = hs + M * M;                      // rows_per_block x M
  const int rows_per_block = blockDim.x / MP;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) hs[e] = H[e];
  const int rr = threadIdx.x / MP, a = threadIdx.x % MP;
  const int64_t i = (int64_t)blockIdx.x * rows_per_block + rr;
  const bool act = rr < rows_per_block && i < N && a < M;
  if (act) fs[rr * M + a] = F[i * M + a];
  __syncthreads();
  if (!act) return;
  T den = T(0);
  for (int b = 0; b < M; ++b) den = fma(fs[rr * M + b], hs[b * M + a], den);
  const T f = fs[rr * M + a];
  const T v = f * Num[i * M + a] / (den > eps ? den : eps);
  F[i * M + a] = v > T(0) ? v : T(0);
}

template <typename T>
__global__ void elementwise_mu_kernel(T* __restrict__ th, const T* __restrict__ num,
                                      const T* __restrict__ den, int64_t n, T eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T d = den[i];
    const T v = th[i] * num[i] / (d > eps ? d : eps);
    th[i] = v > T(0) ? v : T(0);
  }
}

template <typename T>
__global__ void residual_identity_kernel(const T* __restrict__ M, const T* __restrict__ G,
                                         const T* __restrict__ Dn, int64_t n,
                                         const double* __restrict__ x2, double* trace,
                                         int stride, int* counter) {
  __shared__ double sh[32];
  double mg = 0.0, gd = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double g = (double)G[i];
    mg += (double)M[i] * g;
    gd += g * (double)Dn[i];
  }
  mg = block_sum(mg, sh);
  gd = block_sum(gd, sh);
  if (threadIdx.x == 0) {
    const double xx = *x2;
    double r2 = xx - 2.0 * mg + gd;
    if (r2 < 0.0) r2 = 0.0;
    const int t = *counter;
    trace[(int64_t)t * stride] = sqrt(r2 / xx);
    *counter = t + 1;
  }
}

template <typename T>
__global__ void tensor_stats_kernel(const T* __restrict__ X, int64_t n, double* part) {
  __shared__ double sh[32];
  double s2 = 0.0, bad = 0.0, neg = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)X[i];
    if (!isfinite(v)) {
      bad += 1.0;
    } else {
      s2 += v * v;
      if (v < 0.0) neg += 1.0;
    }
  }
  s2 = block_sum(s2, sh);
  neg = block_sum(neg, sh);
  bad = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = s2;
    part[3 * blockIdx.x + 1] = neg;
    part[3 * blockIdx.x + 2] = bad;
  }
}

__global__ void tensor_stats_final_kernel(const double* __restrict__ part, int nblocks,
                                          double* out) {
  __shared__ double sh[32];
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 3; ++k) s[k] += part[3 * b + k];
  for (int k = 0; k < 3; ++k) {
    const double t = block_sum(s[k], sh);
    if (threadIdx.x == 0) out[k] = t;
  }
}

template <typename T, typename U>
__global__ void convert_kernel(const T* __restrict__ src, U* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (U)src[i];
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 4096) {
  int64_t b = ceil_div(n, threads);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t launch_pair_contract(const T* Y, const T* G, int64_t L, int NI, int MA, int64_t C,
                                 T* out, cudaStream_t s) {
  const size_t smem = (size_t)(L * C) * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit((const void*)pair_contract_kernel<T>, smem);
    if (e != cudaSuccess) return e;
  }
  pair_contract_kernel<T><<<NI, 256, smem, s>>>(Y, G, L, NI, MA, C, out);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor_mu(T* F, const T* Num, const T* H, int64_t N, int M, double eps,
                             cudaStream_t s) {
  const int MP = (M + 31) / 32 * 32;
  const int threads = MP > 256 ? MP : 256;
  const int rows = threads / MP;
  const size_t smem = ((size_t)M * M + (size_t)rows * M) * sizeof(T);
  factor_mu_kernel<T><<<(unsigned)ceil_div(N, rows), threads, smem, s>>>(F, Num, H, N, M, MP,
                                                                          (T)eps);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_elementwise_mu(T* theta, const T* num, const T* den, int64_t n, double eps,
                                  cudaStream_t s) {
  elementwise_mu_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(theta, num, den, n, (T)eps);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_identity(const T* M, const T* G, const T* Dn, int64_t n,
                                     const double* x2, double* trace, int stride, int* counter,
                                     cudaStream_t s) {
  residual_identity_kernel<T><<<1, 1024, 0, s>>>(M, G, Dn, n, x2, trace, stride, counter);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tensor_stats(const T* X, int64_t n, double* part, double* out, cudaStream_t s) {
  const unsigned blocks = grid_for(n, 256, kStatBlocks);
  tensor_stats_kernel<T><<<blocks, 256, 0, s>>>(X, n, part);
  note_launch(s);
  tensor_stats_final_kernel<<<1, 256, 0, s>>>(part, (int)blocks, out);
  note_launch(s);
  return cudaGetLastError();
}

template <typename T, typename U>
cudaError_t launch_convert(const T* src, U* dst, int64_t n, cudaStream_t s) {
  convert_kernel<T, U><<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  note_launch(s);
  return cudaGetLastError();
}

#define NNC_INST(T)                                                                            \
  template cudaError_t launch_pair_contract<T>(const T*, const T*, int64_t, int, int, int64_t,  \
                                               T*, cudaStream_t);                              \
  template cudaError_t launch_factor_mu<T>(T*, const T*, const T*, int64_t, int, double,       \
                                           cudaStream_t);                                      \
  template cudaError_t launch_elementwise_mu<T>(T*, const T*, const T*, int64_t, double,       \
                                                cudaStream_t);                                 \
  template cudaError_t launch_residual_identity<T>(const T*, const T*, const T*, int64_t,      \
                                                   const double*, double*, int, int*,          \
                                                   cudaStream_t);                              \
  template cudaError_t launch_tensor_stats<T>(const T*, int64_t, double*, double*, cudaStream_t);
NNC_INST(float)
NNC_INST(double)
#undef NNC_INST

template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);

}  // namespace nnc
