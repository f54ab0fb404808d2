// Launchers of the SIMT kernels (definitions in ttm.cu, small.cu, nncp.cu,
// residual.cu). T is float or double; every launcher is stream-ordered and
// returns the launch status.
#pragma once

#include "common.cuh"

namespace nnc {

// Mode product on a tensor viewed as (L, J, C) in C order (Appendix A, Def. of
// n-mode multiplication, with A = Fm^T):
//   out[l, q, c] = sum_j Fm[j * fs_j + q * fs_q] * Y[(l * J + j) * C + c]
// out is (L, Q, C). When the launch would not fill the GPU, the J range is
// split over blocks that write partial sums to `split_buf` (capacity
// `split_cap` elements), which a second kernel adds in a fixed order.
template <typename T>
cudaError_t launch_ttm(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                       int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                       cudaStream_t s);

// The same mode product on the tensor cores for float tensors with C > 1,
// C % 4 == 0, Q <= 32 and Y 16-byte aligned (TF32x3 operands on mma.sync,
// FP32-accurate); every other case, and double, goes to launch_ttm.
template <typename T>
cudaError_t launch_ttm_tc(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                          int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                          cudaStream_t s);

// out[i, a] = sum_{l, c} Y[(l * NI + i) * C + c] * G[(l * MA + a) * C + c]
// Y is (L, NI, C), G is (L, MA, C), out is NI x MA (MA <= 64, L C < 2^31). It
// is the product of the mode-n unfoldings unfold_n(Y) unfold_n(G)^T when the
// tensors are viewed with mode n in the middle. The flattened (l, c) range is
// split over blocks when the rows alone would not fill the GPU; the partial
// sums (at most part_cap elements of `part`) are added in split order. With
// parts_out, the sums are left to the consumer: *parts_out = the number of
// partials, in `part` (NI MA apart) when it is above 1, else the result is in out.
template <typename T>
cudaError_t launch_pair_contract(const T* Y, const T* G, int64_t L, int NI, int MA, int64_t C,
                                 T* out, T* part, size_t part_cap, cudaStream_t s,
                                 int* parts_out = nullptr);

// out[i] = sum_{p < splits} part[p n + i], p in order.
template <typename T>
cudaError_t launch_reduce_splits(const T* part, int splits, int64_t n, T* out, cudaStream_t s);

// F[i, a] <- max(F[i, a] * Num[i, a] / max(sum_b F[i, b] H[b, a], eps), 0),
// F and Num N x M, H M x M; with parts > 1, Num[i, a] is the sum of the
// partials Num[p N M + i M + a], p = 0 .. parts - 1 added in order.
template <typename T>
cudaError_t launch_factor_mu(T* F, const T* Num, const T* H, int64_t N, int M, double eps,
                             cudaStream_t s, int parts = 1);

// theta <- max(theta * num / max(den, eps), 0), elementwise over n entries.
template <typename T>
cudaError_t launch_elementwise_mu(T* theta, const T* num, const T* den, int64_t n, double eps,
                                  cudaStream_t s);

// trace[(*counter) * stride] = sqrt(max(x2 - 2 <M, G> + <G, Dn>, 0) / x2), FP64
// sums over n core entries (per-block partials in `part`, 2 kIdentityBlocks
// doubles, added in block order); then *counter += 1. `counter` is the pair of
// trace_record (the second int flags the first non-finite entry).
constexpr int kIdentityBlocks = 128;
template <typename T>
cudaError_t launch_residual_identity(const T* M, const T* G, const T* Dn, int64_t n,
                                     const double* x2, double* trace, int stride, int* counter,
                                     double* part, cudaStream_t s);

// One pass over X: sum of squares (FP64) and counts of negative and
// non-finite entries. part holds >= 3 * kStatBlocks doubles, out 3 doubles:
// {sum x^2, #negative, #non-finite}.
constexpr int kStatBlocks = 1024;
template <typename T>
cudaError_t launch_tensor_stats(const T* X, int64_t n, double* part, double* out, cudaStream_t s);

// Per-element conversion: dst = (U)src.
template <typename T, typename U>
cudaError_t launch_convert(const T* src, U* dst, int64_t n, cudaStream_t s);

}  // namespace nnc
