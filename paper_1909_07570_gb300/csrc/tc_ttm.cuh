// Tensor-core passes over X (tc_ttm.cu): BF16, and FP32-accurate TF32x3.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace nnc {
namespace tc {

constexpr int kKindBf16 = 0;
constexpr int kKindTf32x3 = 1;

// Where and how the epilogue writes one pass's FP32 result.
struct TcEpilogue {
  float* out;
  int q;                  // output columns written (m_n)
  // pass X x_3 F3^T: out is rows x q, row r scaled by row_scale[r / rows_per_slice]
  // (row_scale NULL: no scaling)
  int64_t rows;
  int64_t rows_per_slice;
  const float* row_scale;
  // p1_layout 0: out is rows x q, tile row = output row (as above)
  // p1_layout 1 (pass X x_1 F1^T): tile row c = (j, k) of the N2 x kp layout
  //   (kp = padded row length of the operand view); out is q x n2 x n3
  //   (slab = n2 n3)
  // p1_layout 2 (pass X x_1 F1^T): tile row c = (j, k) of the N2 x kp layout;
  //   out has rows (k, j): out[(k n2 + j) q + col]
  int p1_layout;
  int64_t kp, n2, n3, slab;
  // Optional contraction of each tile with the matching rows of a factor F
  // (N2 % 128 == 0, q <= 32, yf_m <= 32). Both passes see tiles of 128 rows
  // (s, j) with j = j0 .. j0 + 127, j0 = 128 (tile % y_nh), y_nh = N2 / 128,
  // s = i (pass X x_3 F3^T) or k (pass X x_1 F1^T with rows (k, j)). The tile
  // writes its share of Y[s] = F^T P[s] (yf_m x q), or of its transpose when
  // y_tr (q x yf_m):
  //   ysh[tile yf_m q + b q + c] = sum_r yf[(j0 + r) yf_m + b] P[(s, j0 + r), c]
  float* ysh;
  const float* yf;
  int yf_m;
  int y_tr;
  int64_t y_nh;
};

// Operands and TMA descriptors of the two passes over a 3-way FP32 X.
//   BF16:   a BF16 copy Xb of X (per-slice power-of-two scales, rows padded to a
//           multiple of 64) and BF16 operands Bt1, Bt3 of F^(1), F^(3).
//   TF32x3: X itself for pass 1, a transposed copy Xt (N2 N3 x N1p, i
//           contiguous; rows (j, k), or (k, j) with p1_kj) so that pass 2 is
//           K-major too, and hi / lo TF32 operands B1hi/B1lo, B3hi/B3lo.
// B operands are [np x k] row-major, zero outside the factor.
struct TcPlan {
  int kind = kKindBf16;
  // Layout of the pass-2 result: false: m1 x N2 x N3; true: rows (k, j),
  // (N3 N2) x m1 (the nnTD sweep's layout).
  bool p1_kj = false;
  int64_t N1 = 0, N2 = 0, N3 = 0;
  int m1 = 0, m3 = 0, kp1 = 0, kp3 = 0, kb3 = 0, np1 = 0, np3 = 0;
  __nv_bfloat16 *Xb = nullptr, *Bt1 = nullptr, *Bt3 = nullptr;
  float *B1hi = nullptr, *B1lo = nullptr, *B3hi = nullptr, *B3lo = nullptr, *Xt = nullptr;
  float *scale = nullptr, *inv_scale = nullptr;
  int* err = nullptr;
  // SMs a pass of at least 8 tiles per SM leaves to kernels that run beside
  // it (the nnTD sweep's small kernels); 0: every SM.
  int reserve_sms = 0;
  CUtensorMap mapA3, mapB3, mapB3lo, mapA1, mapB1, mapB1lo;

  // Builds the operand buffers (BF16: Xb and the scales) from X, stream-ordered.
  // UNSUPPORTED when the shape is outside the path (m_n > 64; TF32x3 also
  // needs N3 % 4 == 0 for its TMA row strides).
  int init(int kind, const float* X, int64_t N1, int64_t N2, int64_t N3, int m1, int m3,
           Scratch& sc, cudaStream_t s, bool p1_kj = false);
  // B operands from the current factor (BF16: F^(1) scaled by s).
  int convert_b3(const float* F3, cudaStream_t s) const;
  int convert_b1(const float* F1, cudaStream_t s) const;
  // P3 = X x_3 F3^T ((N1 N2) x m3, FP32); convert first builds the B operand.
  // With Y1 (y1_fusable(m2) only) the pass also writes the per-tile shares of
  // Y1[i] = F2^T P3[i, :, :] (m2 x m3 each; see TcEpilogue::ysh).
  int pass3(const float* F3, float* P3, cudaStream_t s, bool convert = true,
            const float* F2 = nullptr, int m2 = 0, float* Y1 = nullptr) const;
  bool y1_fusable(int m2) const;
  // P1 = X x_1 F1^T (FP32; m1 x N2 x N3, or rows (k, j) with p1_kj).
  // With Y3 (y3_fusable(m2) only: TF32x3 with p1_kj) the pass also writes the
  // per-tile shares of Y3[k] = P1[k, :, :]^T F2 (m1 x m2 each).
  int pass1(const float* F1, float* P1, cudaStream_t s, bool convert = true,
            const float* F2 = nullptr, int m2 = 0, float* Y3 = nullptr) const;
  bool y3_fusable(int m2) const;
  // Synchronises s and turns a device-side pipeline time-out into NNC_ERR_TIMEOUT.
  int check(cudaStream_t s) const;
};

// Runs the pass kernel's bounded mbarrier wait once, with a limit of `cycles`,
// on a barrier that never completes: NNC_ERR_TIMEOUT when it gives up (the
// expected outcome), NNC_OK if it did not.
int wait_selftest(long long cycles, cudaStream_t s);

}  // namespace tc
}  // namespace nnc
