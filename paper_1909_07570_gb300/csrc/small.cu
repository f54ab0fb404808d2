// Core-sized and factor-sized kernels of an nnTD sweep: unfolding products
// (numerators Num_n and the m_n x m_n matrices of the denominators), the
// multiplicative updates with their nonnegativity projection, the FP64
// residual identity and the one-pass statistics of X.
#include <type_traits>

#include "kernels.cuh"

namespace nnc {
namespace {

// out[i, a] (split s) = sum over k in the split's range of Y[l, i, c] G[l, a, c],
// k = l C + c. A block takes kCtRows rows i and one k range; chunks of kCtK
// consecutive k of both operands are staged in shared memory (consecutive k
// are consecutive c within a row of Y or G, so the loads coalesce when C is
// large). Thread (ty, tx) keeps rows 2 ty, 2 ty + 1 x a = tx + 16 u (u < 4).
constexpr int kCtRows = 32, kCtK = 32, kCtThreads = 256, kCtMaxA = 64;

template <typename T>
__global__ void __launch_bounds__(kCtThreads)
contract_kernel(const T* __restrict__ Y, const T* __restrict__ G, int C, int NI, int MA, int K,
                int k_per_split, T* __restrict__ out) {
  __shared__ T Ys[kCtK][kCtRows + 1];
  __shared__ T Gs[kCtK][kCtMaxA + 1];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * kCtRows;
  const int kbeg = blockIdx.y * k_per_split;
  const int kend = min(K, kbeg + k_per_split);
  const int ty = tid >> 4, tx = tid & 15;
  const int kk = tid & 31, sub = tid >> 5;  // the loads: one k per lane, rows by warp
  T acc[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[r][u] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += kCtK) {
    const int k = k0 + kk;
    const bool kin = k < kend;
    const int l = kin ? k / C : 0;
    const int c = kin ? k - l * C : 0;
#pragma unroll
    for (int r = sub; r < kCtRows; r += kCtThreads / 32) {
      const int i = i0 + r;
      Ys[kk][r] = (kin && i < NI) ? Y[((int64_t)l * NI + i) * C + c] : T(0);
    }
#pragma unroll
    for (int a = sub; a < kCtMaxA; a += kCtThreads / 32)
      Gs[kk][a] = (kin && a < MA) ? G[((int64_t)l * MA + a) * C + c] : T(0);
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < kCtK; ++q) {
      const T y0 = Ys[q][2 * ty], y1 = Ys[q][2 * ty + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T g = Gs[q][tx + 16 * u];
        acc[0][u] = fma(y0, g, acc[0][u]);
        acc[1][u] = fma(y1, g, acc[1][u]);
      }
    }
    __syncthreads();
  }
  T* o = out + (int64_t)blockIdx.y * NI * MA;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int i = i0 + 2 * ty + r;
    if (i >= NI) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int a = tx + 16 * u;
      if (a < MA) o[(int64_t)i * MA + a] = acc[r][u];
    }
  }
}

// Rows of F are updated by one group of M' = roundup(M, 32) threads each; the
// old row is staged in shared memory before any entry of it is overwritten.
// The numerator is the sum of `parts` partial numerators `part_stride` apart,
// added in order p = 0, 1, ... (as reduce_splits_kernel adds them).
template <typename T>
__global__ void factor_mu_kernel(T* __restrict__ F, const T* __restrict__ Num, int parts,
                                 int64_t part_stride, const T* __restrict__ H, int64_t N, int M,
                                 int MP, T eps) {
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
  const T* np = Num + i * M + a;
  T num = np[0];
  int p = 1;
  for (; p + 8 <= parts; p += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = np[(int64_t)(p + u) * part_stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) num += v[u];
  }
  for (; p < parts; ++p) num += np[(int64_t)p * part_stride];
  const T f = fs[rr * M + a];
  const T v = f * num / (den > eps ? den : eps);
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

// Partials of <M, G> and <G, Dn> in FP64: block b sums the entries
// b, b + B, b + 2B, ... of its grid stride (B = blocks x threads).
template <typename T>
__global__ void identity_part_kernel(const T* __restrict__ M, const T* __restrict__ G,
                                     const T* __restrict__ Dn, int64_t n, double* part) {
  __shared__ double sh[32];
  double mg = 0.0, gd = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double g = (double)G[i];
    mg += (double)M[i] * g;
    gd += g * (double)Dn[i];
  }
  mg = block_sum(mg, sh);
  gd = block_sum(gd, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = mg;
    part[2 * blockIdx.x + 1] = gd;
  }
}

// The partials added in block order, then the trace entry.
__global__ void identity_final_kernel(const double* __restrict__ part, int nb,
                                      const double* __restrict__ x2, double* trace, int stride,
                                      int* counter) {
  __shared__ double sh[32];
  double mg = 0.0, gd = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    mg += part[2 * b];
    gd += part[2 * b + 1];
  }
  mg = block_sum(mg, sh);
  gd = block_sum(gd, sh);
  if (threadIdx.x == 0) {
    const double xx = *x2;
    double r2 = xx - 2.0 * mg + gd;
    const bool finite = isfinite(r2);
    if (r2 < 0.0) r2 = 0.0;
    trace_record(counter, trace, stride, sqrt(r2 / xx), finite);
  }
}

template <typename T>
__global__ void tensor_stats_kernel(const T* __restrict__ X, int64_t n, double* part) {
  __shared__ double sh[32];
  double s2 = 0.0;
  unsigned neg = 0, bad = 0;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t head = 0;  // elements handled by the vector loop
  if constexpr (std::is_same<T, float>::value) {
    // GB300's FP64 rate is far below its FP32 rate: the squares of each
    // 8-element chunk (two 16-byte loads) are added in FP32, rounded to
    // nearest, and only the chunk sums in FP64. The rounding errors are
    // unbiased, so their sum over the tensor stays far below FP64's own.
    if ((reinterpret_cast<uintptr_t>(X) & 15) == 0) {
      const float4* x4 = reinterpret_cast<const float4*>(X);
      const int64_t nv = n / 8;
      for (int64_t v = tid; v < nv; v += nth) {
        const float4 a = x4[2 * v], b = x4[2 * v + 1];
        const float e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        float c = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float x = e[t];
          if (!(fabsf(x) <= 3.402823466e38f)) {
            ++bad;
          } else {
            c = fmaf(x, x, c);
            neg += x < 0.f;
          }
        }
        if (c <= 3.402823466e38f) {
          s2 += (double)c;
        } else {  // the FP32 squares overflowed (entries beyond 1.8e19): FP64
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (fabsf(e[t]) <= 3.402823466e38f) s2 += (double)e[t] * (double)e[t];
        }
      }
      head = nv * 8;
    }
  }
  for (int64_t i = head + tid; i < n; i += nth) {
    const double v = (double)X[i];
    if (!isfinite(v)) {
      ++bad;
    } else {
      s2 += v * v;
      neg += v < 0.0;
    }
  }
  s2 = block_sum(s2, sh);
  const double dneg = block_sum((double)neg, sh);
  const double dbad = block_sum((double)bad, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = s2;
    part[3 * blockIdx.x + 1] = dneg;
    part[3 * blockIdx.x + 2] = dbad;
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
                                 T* out, T* part, size_t part_cap, cudaStream_t s,
                                 int* parts_out) {
  if (L < 1 || NI < 1 || MA < 1 || MA > kCtMaxA || C < 1 || L * C > 2147483647LL)
    return cudaErrorInvalidValue;
  const int K = (int)(L * C);
  const int64_t row_tiles = ceil_div((int64_t)NI, kCtRows);
  if (row_tiles > 65535) return cudaErrorInvalidValue;
  // Splits of k: about two blocks per SM, at least 4 chunks per split, and
  // the partials within the scratch.
  int64_t splits = ceil_div(2LL * device_sm_count(), row_tiles);
  const int64_t by_k = K / (4 * kCtK);
  const int64_t by_cap = part ? (int64_t)(part_cap / ((size_t)NI * MA)) : 1;
  if (splits > by_k) splits = by_k;
  if (splits > by_cap) splits = by_cap;
  if (splits < 1) splits = 1;
  const int per = (int)(ceil_div(ceil_div((int64_t)K, splits), kCtK) * kCtK);
  splits = ceil_div((int64_t)K, per);
  T* dst = splits > 1 ? part : out;
  contract_kernel<T><<<dim3((unsigned)row_tiles, (unsigned)splits), kCtThreads, 0, s>>>(
      Y, G, (int)C, NI, MA, K, per, dst);
  note_launch(s);
  if (parts_out) *parts_out = (int)splits;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1 || parts_out) return e;
  return launch_reduce_splits<T>(part, (int)splits, (int64_t)NI * MA, out, s);
}

template <typename T>
cudaError_t launch_factor_mu(T* F, const T* Num, const T* H, int64_t N, int M, double eps,
                             cudaStream_t s, int parts) {
  if (parts < 1) return cudaErrorInvalidValue;
  const int MP = (M + 31) / 32 * 32;
  const int threads = MP > 256 ? MP : 256;
  const int rows = threads / MP;
  const size_t smem = ((size_t)M * M + (size_t)rows * M) * sizeof(T);
  factor_mu_kernel<T><<<(unsigned)ceil_div(N, rows), threads, smem, s>>>(
      F, Num, parts, N * M, H, N, M, MP, (T)eps);
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
                                     double* part, cudaStream_t s) {
  const unsigned nb = grid_for(n, 256, kIdentityBlocks);
  identity_part_kernel<T><<<nb, 256, 0, s>>>(M, G, Dn, n, part);
  note_launch(s);
  identity_final_kernel<<<1, 256, 0, s>>>(part, (int)nb, x2, trace, stride, counter);
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
                                               T*, T*, size_t, cudaStream_t, int*);            \
  template cudaError_t launch_factor_mu<T>(T*, const T*, const T*, int64_t, int, double,       \
                                           cudaStream_t, int);                                 \
  template cudaError_t launch_elementwise_mu<T>(T*, const T*, const T*, int64_t, double,       \
                                                cudaStream_t);                                 \
  template cudaError_t launch_residual_identity<T>(const T*, const T*, const T*, int64_t,      \
                                                   const double*, double*, int, int*, double*, \
                                                   cudaStream_t);                              \
  template cudaError_t launch_tensor_stats<T>(const T*, int64_t, double*, double*, cudaStream_t);
NNC_INST(float)
NNC_INST(double)
#undef NNC_INST

template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);

}  // namespace nnc
