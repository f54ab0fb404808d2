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
// The scratch of residual evaluations, taken once (residual_prepare) and
// reused by any number of residual_run calls, which allocate nothing.
template <typename T>
struct ResidualWork {
  T* U = nullptr;           // model rows, N_1 ... N_{d-1} x (m_d or r)
  T* tmp[2] = {nullptr, nullptr};  // intermediate mode products
  double* part = nullptr;   // per-block partial sums
  int64_t nblocks = 0;
};
template <typename T>
int residual_prepare(int d, const int64_t* dims, int model, const int* m, int r, Scratch& sc,
                     ResidualWork<T>* w);
// As residual_device with prepared scratch; out2 (2 doubles) and rel_out
// (||X - X_hat|| / ||X||, one double) are device pointers, either may be NULL.
template <typename T>
int residual_run(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                 const T* const* factors, const T* G, const ResidualWork<T>& w, double* out2,
                 double* rel_out, cudaStream_t s);

template <typename T>
int residual_device(const T* X, int d, const int64_t* dims, int model, const int* m, int r,
                    const T* const* factors, const T* G, double* out2, Scratch& sc,
                    cudaStream_t s);

}  // namespace nnc
