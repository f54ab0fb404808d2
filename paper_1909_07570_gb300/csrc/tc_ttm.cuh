// Tensor-core passes over X for the BF16 path (tc_ttm.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace nnc {
namespace tc {

// Where and how the epilogue writes one pass's FP32 result.
struct TcEpilogue {
  float* out;
  int q;                  // output columns written (m_n)
  // pass X x_3 F3^T: out is rows x q, row r scaled by row_scale[r / rows_per_slice]
  int64_t rows;
  int64_t rows_per_slice;
  const float* row_scale;
  // pass X x_1 F1^T: tile row c = (j, k) of the padded N2 x kp layout; out is
  // q x n2 x n3 (slab = n2 n3)
  int64_t kp, n2, n3, slab;
};

// The BF16 copy of a 3-way FP32 X with its slice scales, the BF16 operand
// buffers of F^(3)T and F^(1)T, and the TMA descriptors of both passes.
struct TcPlan {
  int64_t N1 = 0, N2 = 0, N3 = 0;
  int m1 = 0, m3 = 0, kp1 = 0, kp3 = 0, np1 = 0, np3 = 0;
  __nv_bfloat16 *Xb = nullptr, *Bt1 = nullptr, *Bt3 = nullptr;
  float *scale = nullptr, *inv_scale = nullptr;
  int* err = nullptr;
  CUtensorMap mapA3, mapB3, mapA1, mapB1;

  // Builds Xb and the scales from X (stream-ordered). UNSUPPORTED when the
  // shape is outside the path (m_n > 64, or a factor too long for one CTA's
  // shared memory).
  int init(const float* X, int64_t N1, int64_t N2, int64_t N3, int m1, int m3, Scratch& sc,
           cudaStream_t s);
  // P3 = X x_3 F3^T ((N1 N2) x m3, FP32). With convert, Bt3 is first built
  // from F3; without, Bt3 already holds bf16(F3^T) (written by the sweep).
  int pass3(const float* F3, float* P3, cudaStream_t s, bool convert = true) const;
  // P1 = X x_1 F1^T (m1 x N2 x N3, FP32); Bt1 as above, from diag(s) F1.
  int pass1(const float* F1, float* P1, cudaStream_t s, bool convert = true) const;
  // Synchronises s and turns a device-side pipeline time-out into NNC_ERR_TIMEOUT.
  int check(cudaStream_t s) const;
};

}  // namespace tc
}  // namespace nnc
