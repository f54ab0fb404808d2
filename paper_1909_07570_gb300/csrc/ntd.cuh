// nnTD of a 3-way tensor (ntd.cu): the body of ntd_fit.
#pragma once

#include "common.cuh"

namespace nnc {

// FP64 (T = double) and FP32 (T = float) paths. Arguments as ntd_fit with
// d = 3, already validated. tensor_cores (float only): TF32x3 passes where the
// shape allows, else SIMT.
template <typename T>
int ntd_fit3(const T* X, const int64_t* dims, const int* m, const nnc_opts* o, T* const* F, T* G,
             double* trace, double* rel_err, bool tensor_cores, cudaStream_t s);

// NNC_BF16_REFINE path; *refined_from (may be NULL) gets the index of the
// first FP32 refinement sweep (iters when there was none).
int ntd_fit3_bf16(const float* X, const int64_t* dims, const int* m, const nnc_opts* o,
                  float* const* F, float* G, double* trace, double* rel_err, int* refined_from,
                  cudaStream_t s);

}  // namespace nnc
