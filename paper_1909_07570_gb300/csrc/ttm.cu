// SIMT mode products (n-mode multiplication, Appendix A) used by the FP32 and
// FP64 paths: the two passes over X of every sweep and all the small
// contractions around them.
//
// A tensor is viewed as (L, J, C) with J the contracted mode:
//   out[l, q, c] = sum_j Fm[j, q] * Y[l, j, c]
// Two kernels cover the two memory patterns:
//   * ttm_rows (C == 1): J is the contiguous axis (e.g. X x_3 F^(3)T). A block
//     stages a BM x 32 tile of Y and a 32 x QP slice of Fm in shared memory;
//     each thread keeps TR rows x QP outputs in registers.
//   * ttm_cols (C > 1): J is strided (e.g. X x_1 F^(1)T). Each thread owns TC
//     flattened (l, c) columns, streams them along j with coalesced loads and
//     keeps QP outputs per column in registers; Fm rows are broadcast from
//     shared memory.
// Both accumulate in T and, when one pass would not fill the GPU, split J
// across blocks; partial sums are then added in split order (deterministic).
#include "kernels.cuh"

namespace nnc {
namespace {

constexpr int kRowsThreads = 128;
// K-chunk of ttm_rows: 32 for float, 16 for double (static shared memory < 48 KB).
template <typename T>
__host__ __device__ constexpr int rows_bk() { return sizeof(T) == 4 ? 32 : 16; }
constexpr int kColsThreads = 256;
constexpr int kColsBJ = 32;

template <typename T, int QP, int TR>
__global__ void __launch_bounds__(kRowsThreads)
ttm_rows_kernel(const T* __restrict__ Y, int64_t R, int K, int k_per_split,
                const T* __restrict__ Fm, int64_t fs_k, int64_t fs_q, int Q,
                T* __restrict__ out) {
  constexpr int BM = kRowsThreads * TR;
  constexpr int BK = rows_bk<T>();
  __shared__ T Xs[BM][BK + 1];
  __shared__ __align__(16) T Fs[BK][QP];

  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * BM;
  const int kbeg = blockIdx.y * k_per_split;
  const int kend = min(K, kbeg + k_per_split);

  T acc[TR][QP];
#pragma unroll
  for (int t = 0; t < TR; ++t)
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[t][q] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BM * BK; e += kRowsThreads) {
      const int rr = e / BK, kk = e % BK;
      const int64_t r = r0 + rr;
      const int k = k0 + kk;
      Xs[rr][kk] = (r < R && k < kend) ? Y[r * K + k] : T(0);
    }
    for (int e = tid; e < BK * QP; e += kRowsThreads) {
      const int kk = e / QP, q = e % QP;
      const int k = k0 + kk;
      Fs[kk][q] = (q < Q && k < kend) ? Fm[k * fs_k + q * fs_q] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      T x[TR];
#pragma unroll
      for (int t = 0; t < TR; ++t) x[t] = Xs[tid + t * kRowsThreads][kk];
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const T f = Fs[kk][q];
#pragma unroll
        for (int t = 0; t < TR; ++t) acc[t][q] = fma(x[t], f, acc[t][q]);
      }
    }
    __syncthreads();
  }

  T* o = out + (int64_t)blockIdx.y * R * Q;
#pragma unroll
  for (int t = 0; t < TR; ++t) {
    const int64_t r = r0 + tid + t * kRowsThreads;
    if (r < R) {
#pragma unroll
      for (int q = 0; q < QP; ++q)
        if (q < Q) o[r * Q + q] = acc[t][q];
    }
  }
}

template <typename T, int QP, int TC>
__global__ void __launch_bounds__(kColsThreads)
ttm_cols_kernel(const T* __restrict__ Y, int64_t L, int J, int64_t C, int j_per_split,
                const T* __restrict__ Fm, int64_t fs_j, int64_t fs_q, int Q,
                T* __restrict__ out) {
  constexpr int BJ = kColsBJ;
  __shared__ __align__(16) T Fs[BJ][QP];

  const int64_t ncols = L * C;
  const int64_t base = (int64_t)blockIdx.x * (kColsThreads * TC) + threadIdx.x;
  const int jbeg = blockIdx.y * j_per_split;
  const int jend = min(J, jbeg + j_per_split);

  const T* y[TC];
  int64_t col_l[TC], col_c[TC];
  bool active[TC];
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int64_t g = base + (int64_t)t * kColsThreads;
    active[t] = g < ncols;
    const int64_t gg = active[t] ? g : 0;
    col_l[t] = gg / C;
    col_c[t] = gg % C;
    y[t] = Y + col_l[t] * (int64_t)J * C + col_c[t];
  }

  T acc[TC][QP];
#pragma unroll
  for (int t = 0; t < TC; ++t)
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[t][q] = T(0);

  for (int j0 = jbeg; j0 < jend; j0 += BJ) {
    for (int e = threadIdx.x; e < BJ * QP; e += kColsThreads) {
      const int jj = e / QP, q = e % QP;
      const int j = j0 + jj;
      Fs[jj][q] = (q < Q && j < jend) ? Fm[j * fs_j + q * fs_q] : T(0);
    }
    __syncthreads();
    const int jn = min(BJ, jend - j0);
#pragma unroll 4
    for (int jj = 0; jj < jn; ++jj) {
      T v[TC];
#pragma unroll
      for (int t = 0; t < TC; ++t) v[t] = active[t] ? y[t][(int64_t)(j0 + jj) * C] : T(0);
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const T f = Fs[jj][q];
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[t][q] = fma(f, v[t], acc[t][q]);
      }
    }
    __syncthreads();
  }

  T* o = out + (int64_t)blockIdx.y * L * Q * C;
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    if (!active[t]) continue;
    T* ot = o + col_l[t] * Q * C + col_c[t];
#pragma unroll
    for (int q = 0; q < QP; ++q)
      if (q < Q) ot[(int64_t)q * C] = acc[t][q];
  }
}

template <typename T>
__global__ void reduce_splits_kernel(const T* __restrict__ part, int splits, int64_t n,
                                     T* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = part[i];
    for (int p = 1; p < splits; ++p) s += part[(int64_t)p * n + i];
    out[i] = s;
  }
}

// Number of J-splits so that about two blocks per SM are in flight, bounded by
// the scratch capacity and by one 32-wide chunk of J per split.
int choose_splits(int64_t blocks, int J, int64_t out_elems, size_t split_cap, int chunk,
                  int* per_split) {
  const int64_t target = 2LL * device_sm_count();
  int splits = 1;
  if (blocks < target && J >= 2 * chunk && split_cap > 0) {
    int64_t want = ceil_div(target, blocks);
    int64_t by_j = J / chunk;
    int64_t by_cap = (int64_t)(split_cap / (size_t)out_elems);
    int64_t s = want;
    if (s > by_j) s = by_j;
    if (s > by_cap) s = by_cap;
    if (s > 1) splits = (int)s;
  }
  int per = (int)ceil_div(J, splits);
  per = (int)(ceil_div(per, chunk) * chunk);
  *per_split = per;
  return (int)ceil_div(J, per);
}

template <typename T, int QP>
cudaError_t ttm_dispatch(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                         int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                         cudaStream_t s) {
  const int64_t out_elems = L * Q * C;
  int per = J, splits = 1;
  if (C == 1) {
    constexpr int TR = (sizeof(T) == 4 && QP <= 32) ? 2 : 1;
    constexpr int BM = kRowsThreads * TR;
    const int64_t blocks = ceil_div(L, BM);
    splits = choose_splits(blocks, J, out_elems, split_cap, rows_bk<T>(), &per);
    T* dst = splits > 1 ? split_buf : out;
    dim3 grid((unsigned)blocks, (unsigned)splits);
    ttm_rows_kernel<T, QP, TR><<<grid, kRowsThreads, 0, s>>>(Y, L, J, per, Fm, fs_j, fs_q, Q, dst);
    note_launch(s);
  } else {
    const int64_t ncols = L * C;
    const bool wide = (QP <= 32) && ceil_div(ncols, 2 * kColsThreads) >= 2LL * device_sm_count();
    if (wide) {
      const int64_t blocks = ceil_div(ncols, 2 * kColsThreads);
      splits = choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
      T* dst = splits > 1 ? split_buf : out;
      dim3 grid((unsigned)blocks, (unsigned)splits);
      ttm_cols_kernel<T, QP, 2><<<grid, kColsThreads, 0, s>>>(Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
      note_launch(s);
    } else {
      const int64_t blocks = ceil_div(ncols, kColsThreads);
      splits = choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
      T* dst = splits > 1 ? split_buf : out;
      dim3 grid((unsigned)blocks, (unsigned)splits);
      ttm_cols_kernel<T, QP, 1><<<grid, kColsThreads, 0, s>>>(Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
      note_launch(s);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t blocks = ceil_div(out_elems, 256) < 4096 ? ceil_div(out_elems, 256) : 4096;
  reduce_splits_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(split_buf, splits, out_elems, out);
  note_launch(s);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_ttm(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                       int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                       cudaStream_t s) {
  if (L <= 0 || J <= 0 || C <= 0 || Q <= 0) return cudaErrorInvalidValue;
  if (Q <= 8) return ttm_dispatch<T, 8>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 16) return ttm_dispatch<T, 16>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 32) return ttm_dispatch<T, 32>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 64) return ttm_dispatch<T, 64>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_reduce_splits(const T* part, int splits, int64_t n, T* out, cudaStream_t s) {
  const int64_t blocks = ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096;
  reduce_splits_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(part, splits, n, out);
  note_launch(s);
  return cudaGetLastError();
}

template cudaError_t launch_reduce_splits<float>(const float*, int, int64_t, float*,
                                                 cudaStream_t);
template cudaError_t launch_reduce_splits<double>(const double*, int, int64_t, double*,
                                                  cudaStream_t);
template cudaError_t launch_ttm<float>(const float*, int64_t, int, int64_t, const float*, int64_t,
                                       int64_t, int, float*, float*, size_t, cudaStream_t);
template cudaError_t launch_ttm<double>(const double*, int64_t, int, int64_t, const double*,
                                        int64_t, int64_t, int, double*, double*, size_t,
                                        cudaStream_t);

}  // namespace nnc
