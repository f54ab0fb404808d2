// Differentiation form of the lifted loss (lifted.cu).
#pragma once

#include "common.cuh"

namespace nnc {

// Gradients of L = 1/2 ||X - I x_n F^(n) B^(n)||^2 wrt every F^(n) (into gF)
// and B^(n) (into gB), and L in FP64 (host, optional). gF == nullptr: the loss
// only (one pass over X). d = 3 or 4, m_n <= 64, r <= 64.
template <typename T>
int lifted_grad(const T* X, int d, const int64_t* dims, const int* m, int r, bool tensor_cores,
                T* const* F, T* const* B, T* const* gF, T* const* gB, double* loss,
                cudaStream_t s);

// `steps` block projected-gradient steps on F and B in place; trace (device,
// `steps` doubles, optional) gets L after each step, loss (host, optional) the
// last one.
template <typename T>
int lifted_pg_fit(const T* X, int d, const int64_t* dims, const int* m, int r, bool tensor_cores,
                  int steps, T* const* F, T* const* B, double* trace, double* loss,
                  cudaStream_t s);

// nnCPD of X itself (Alg. 2, first step): `iters` MU sweeps on the CP factors
// A^(n) (dims[n] x r) in place; trace (device, optional) and rel_err (host,
// optional) get ||X - I x_k A^(k)|| / ||X||: the trace from the FP64 identity
// (exact_every > 0: every exact_every-th entry and the last from an explicit
// FP64 pass), rel_err from an explicit pass.
template <typename T>
int nncp_tensor_fit(const T* X, int d, const int64_t* dims, int r, bool tensor_cores, int iters,
                    double eps, int exact_every, T* const* A, double* trace, double* rel_err,
                    cudaStream_t s);

// nnTD of a d-way X (d = 3 or 4) by `iters` MU sweeps (Alg. 1, first step):
// F^(n) (dims[n] x m[n]) and G in place; trace (device, optional) gets the
// relative error after each sweep from the FP64 identity, rel_err (host,
// optional) the final one from an explicit pass over X.
template <typename T>
int ntd_fit_nway(const T* X, int d, const int64_t* dims, const int* m, bool tensor_cores,
                 int iters, double eps, T* const* F, T* G, double* trace, double* rel_err,
                 cudaStream_t s);

// NMF A ~ F B by `iters` MU iterations (Alg. 2, second step), F (N x m) and
// B (m x r) in place; trace / rel_err get ||A - F B|| / ||A||.
template <typename T>
int nmf_fit(const T* A, int64_t N, int r, int m, int iters, double eps, T* F, T* B,
            double* trace, double* rel_err, cudaStream_t s);

}  // namespace nnc
