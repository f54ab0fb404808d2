// Fused kernels of one nnTD sweep (sweep.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace nnc {

// One factor update: Y_r by a small GEMM over the slab r of a pass result,
// then Num[r, :] from Y_r and the core, then the MU step on row r of F.
template <typename T>
struct UpdArgs {
  // p_first == 0: Y_r[u, c] = sum_{t < len} Fc[t, u] P[r prow + t pstride + c]
  // p_first != 0: Y_r[u, c] = sum_{t < len} P[r prow + t pstride + u] Fc[t, c]
  // (u < mu, c < mc; Fc is len x (mu or mc), row-major)
  const T* P;
  int64_t prow, pstride;
  const T* Fc;
  int len;      // contraction length
  int mu, mc;   // Y_r is mu x mc
  int p_first;
  // Optional: Y_r given as the sum of nparts shares Ypart[(r nparts + h) mu mc ..]
  // (h = 0 .. nparts - 1, added in that order) instead of the GEMM.
  const T* Ypart;
  int nparts;
  // Num[r, v] = <Y_r, Gn[v, :]> with Gn the core laid out (m_n, u, c)
  const T* Gn;
  // MU on F (nrows x mv) with Den = F H (H mv x mv)
  T* F;
  int64_t nrows;
  int mv;
  const T* H;
  double eps;
  T* Yout;  // optional: Y_r stored at Yout[r mu mc ..]
  // Optional operand of the next tensor-core pass, entry [v bt_ld + r] for
  // F[r, v] (times bt_scale[r] if given): BF16 (bt) or the TF32 pair (bhi, blo).
  __nv_bfloat16* bt;
  float* bhi;
  float* blo;
  int64_t bt_ld;
  const float* bt_scale;
  int* gate_out;  // optional: set to 1 (mode 3: the sweep's core update is pending)
  // Split update: launch_upd12 with num_only stores Num (nrows x mv) in `num` and
  // leaves F alone; mu_rows then applies the MU step from `num` and H (the
  // numerator does not need H, so the two can run beside the kernel forming H).
  int num_only;
  T* num;
  // FP32 only: the GEMM on the tensor cores when the shape allows it (mu, mc
  // <= 32, 16-byte aligned rows): 1 with TF32 operands, 3 with each operand
  // split into two TF32 parts (FP32-accurate); 0 on the SIMT pipes. Its
  // operands arrive through the TMA unit; a copy that has not arrived after
  // about 2 s sets *err (required for this form) and the block gives up.
  int tc;
  int* err;
  // The tensor-core form's Y_r (nrows x mu mc), from its GEMM to its
  // numerator kernel; Yout (where Y is kept) may serve.
  T* ybuf;
};

// H_n = unfold_n(G x_u S_u x_v S_v) unfold_n(G)^T, one block per index p of mode n.
// Gn is the core laid out (m_n, u, v): slice p is the contiguous U x V block p.
// Each Gram comes either ready (su / sv) or is formed from its factor
// (fu: nu x mu, fv: nv x mv). The W slices go to Wout[p w_sp + u w_su + v w_sv].
template <typename T>
struct HArgs {
  const T* Gn;
  int mp, mu, mv;
  int64_t w_sp, w_su, w_sv;
  const T* su;
  const T* fu;
  int64_t nu;
  const T* sv;
  const T* fv;
  int64_t nv;
  T* su_out;            // optional: the Gram formed from fu (written by block 0)
  T* sv_out;
  T* H;                 // mp x mp
  T* Wout;              // optional: the W slices, laid out like G
  // FP32 only: the Gram on the tensor cores (UpdArgs::tc's values) when the
  // shape allows it (mp, mu, mv <= 32, the factor's rows 16-byte aligned);
  // err as UpdArgs::err (required for that form).
  int tc;
  int* err;
};

template <typename T>
struct CoreArgs {
  T* G;
  T* G2;                // out: G permuted to (m2, m1, m3)
  T* G3;                // out: G permuted to (m3, m1, m2)
  const T* Y3;          // X x_1 F1^T x_2 F2^T laid out (N3, m1, m2)
  T* Mout;              // M = Y3 x_3 F3^T, laid out like G
  const T* W3;          // G x_1 S1 x_2 S2
  const T* S1;
  const T* S2;
  const T* F3;          // S3 = F3^T F3 is formed here
  int64_t n3;
  T* S3_out;
  T* W1;                // out: G_new x_2 S2 x_3 S3
  T* H1;                // out: unfold_1(W1) unfold_1(G_new)^T
  double* dots;         // m1 scratch
  int* done;            // block counter of core_b, 0 between sweeps
  // 1 when a sweep's core update is pending (set by the mode-3 update of that
  // sweep); the core kernels do nothing while it is 0 and core_b clears it.
  int* gate;
  const double* x2;
  double* trace;
  int trace_stride;
  int* counter;         // trace_record pair: entries so far, first non-finite sweep
  int m1, m2, m3;
  double eps;
  // FP32 only: S3 and M on the tensor cores (UpdArgs::tc's values) when the
  // shape allows it (m <= 32, m2 and m3 multiples of 4); err as UpdArgs::err.
  int tc;
  int* err;
};
template <typename T>
int launch_upd12(const UpdArgs<T>& a, cudaStream_t s);
// The tensor-core form of an update in its two parts (launch_upd12 runs both
// when upd_tc_form(a)): launch_upd_gemm forms Y_r into a.ybuf (not with
// a.Ypart); launch_upd_num forms the numerators from a.ybuf or the shares
// a.Ypart and takes the MU step (num_only: stores the numerators).
bool upd_tc_form(const UpdArgs<float>& a);
int launch_upd_gemm(const UpdArgs<float>& a, cudaStream_t s);
int launch_upd_num(const UpdArgs<float>& a, cudaStream_t s);
template <typename T>
int launch_hmat(const HArgs<T>& a, cudaStream_t s);
// F[r] <- MU(F[r], num[r], F[r] H) for every row, with the operand writes and
// gate of UpdArgs (fields P, Fc, Gn, Ypart, Yout unused).
template <typename T>
int launch_mu_rows(const UpdArgs<T>& a, cudaStream_t s);
// P1 rows (k, j): out[(k N2 + j) m1 + a] = in[(a N2 + j) N3 + k].
template <typename T>
int launch_p1_rows(const T* in, int m1, int64_t N2, int64_t N3, T* out, cudaStream_t s);
template <typename T>
int launch_core(const CoreArgs<T>& a, cudaStream_t s);
template <typename T>
int launch_gram(const T* F, int64_t N, int m, T* S, cudaStream_t s);
template <typename T>
int launch_permute_core(const T* G, int m1, int m2, int m3, T* G2, T* G3, cudaStream_t s);

}  // namespace nnc
