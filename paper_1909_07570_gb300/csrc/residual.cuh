// Launchers of the lift and of the one-pass residual (residual.cu).
#pragma once

#include "common.cuh"

namespace nnc {

// A = F B with F N x M, B M x r, A N x r (row-major).
template <typename T>
cudaError_t launch_lift(const T* F, const T* B, int64_t N, int M, int r, T* A, cudaStream_t s);

// out2[0] = ||X - X_hat||_F^2, out2[1] = ||X||_F^2 (device, FP64) for a d-way
// X (d = 3 or 4); model 0 = Tucker (factors F, core G, multirank m), 1 = CP
// (factors A, rank r). Scratch comes from `sc`; the model rows U take
// N_1 ... N_{d-1} x (m_d or r) entries of it.
template <typename T>
int residual_device(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                    const T* const* factors, const T* G, double* out2, Scratch& sc,
                    cudaStream_t s);

}  // namespace nnc
