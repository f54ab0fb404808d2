/*
 * nncandelinc.h - C ABI of the GB300 nnCANDELINC library (libnncandelinc.so).
 *
 * nnCANDELINC (arXiv 1909.07570) approximates a nonnegative d-way tensor X by
 * the lifted model I x_1 F^(1)B^(1) x_2 ... x_d F^(d)B^(d) (Eq. nnCANDELINC,
 * Sec. 4). Alg. 1 (Sec. 4.1) computes it in two steps, nnTD of X followed by
 * nnCPD of the Tucker core; the lift A^(i) = F^(i) B^(i) is the substitution
 * in the proof of Lemma "rank and min exists" (Sec. 2.1).
 *
 * Conventions shared by every call:
 *  - Tensors are dense and C-ordered (the last index is contiguous); index 0
 *    is mode 1 of the paper. Matrices are row-major.
 *  - F^(n) is dims[n] x m[n], G is m[0] x ... x m[d-1], B^(n) is m[n] x r,
 *    A^(n) is dims[n] x r.
 *  - Array pointers (X, F, G, B, A, traces) are DEVICE pointers owned by the
 *    caller; arrays of pointers (F, B, A, factors) and shape arrays (dims, m)
 *    are HOST arrays. Pointers marked "host" are host memory.
 *  - The element type follows `precision`: double for NNC_FP64, float for
 *    NNC_FP32 and NNC_BF16_REFINE (the BF16 copy of X is made internally).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *    stream-ordered. A call returns after its host outputs are written; it
 *    synchronises `stream` only when it has host outputs to write.
 *  - Scratch memory is taken from the stream-ordered allocator
 *    (cudaMallocAsync) on `stream` and released before the call returns.
 *  - Every call returns NNC_OK (0) or a negative NNC_ERR_* code; on error the
 *    caller's arrays may hold partial results. nnc_status_string() names it.
 *  - Update rule: multiplicative updates with a Gauss-Seidel order, guarded
 *    denominators max(den, eps) and a projection max(., 0) (see ntd_fit).
 */
#ifndef NNCANDELINC_H
#define NNCANDELINC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NNC_OK 0
#define NNC_ERR_INVALID_ARG (-1)    /* bad shape, rank, pointer or option      */
#define NNC_ERR_NEGATIVE_INPUT (-2) /* X holds a negative entry                */
#define NNC_ERR_NONFINITE (-3)      /* X holds NaN/Inf, or a result overflowed */
#define NNC_ERR_CUDA (-4)           /* a CUDA runtime call failed              */
#define NNC_ERR_ALLOC (-5)          /* scratch allocation failed               */
#define NNC_ERR_UNSUPPORTED (-6)    /* valid request this build does not serve */
#define NNC_ERR_TIMEOUT (-7)        /* a bounded device-side wait ran out      */

typedef enum {
  NNC_FP64 = 0,        /* double storage and arithmetic (SIMT)               */
  NNC_FP32 = 1,        /* float storage, FP32-accurate arithmetic: the two
                          passes over X per sweep run on the tensor cores as
                          three TF32 products per term (hi*hi + hi*lo + lo*hi
                          of exact TF32 splits, FP32 accumulation); shapes the
                          tensor-core path cannot take (N3 % 4 != 0) run the
                          SIMT passes                                        */
  NNC_BF16_REFINE = 2, /* float storage; the passes over X use a BF16 copy of
                          X on the tensor cores (FP32 accumulation), then the
                          last `refine_iters` sweeps are NNC_FP32 sweeps     */
  NNC_FP32_SIMT = 3    /* as NNC_FP32 with every pass on FP32 FFMA (SIMT)    */
} nnc_precision;

typedef struct {
  int iters;         /* number of MU sweeps, >= 0                          */
  int refine_iters;  /* NNC_BF16_REFINE only: the last refine_iters of the
                        iters sweeps run in FP32 (0 <= refine_iters <= iters) */
  double eps;        /* denominator guard, > 0 (1e-12 in the tests)         */
  int exact_every;   /* ntd_fit (d = 3) and nncp_tensor_fit, with a trace
                        (other calls ignore it):
                        0, or k > 0: after every k-th sweep and after the
                        last, the sweep's trace entry is the relative error
                        of one explicit pass over X with FP64 sums instead of
                        the residual identity (exact near convergence, where
                        the identity cancels; one pass over X per entry)     */
  double refine_tol; /* NNC_BF16_REFINE with exact_every > 0: 0, or tau > 0:
                        the BF16 sweeps also end, and the FP32 refinement
                        sweeps begin, at the first exact checkpoint whose
                        relative decrease since the previous one is below tau
                        times the largest such decrease so far in the fit
                        (progress has slowed to that fraction of its peak);
                        the host reads each checkpoint (one synchronisation
                        per checkpoint). nnc_last_refine_sweep() tells where
                        the switch came                                      */
} nnc_opts;

/*
 * ntd_fit - nonnegative Tucker decomposition X ~ G x_1 F^(1) ... x_d F^(d)
 * (Alg. 1, step 1; model Eq. TD:matrix-format with F, G >= 0, Sec. 3).
 *
 * Runs opts->iters sweeps. A sweep updates F^(1), ..., F^(d) and then G, each
 * by theta <- max(theta * Num / max(Den, eps), 0), where Den - Num is the
 * gradient of 1/2 ||X - X_hat||_F^2 wrt theta:
 *   Num_n = unfold_n(X x_{k!=n} F^(k)T) unfold_n(G)^T
 *   Den_n = F^(n) unfold_n(G x_{k!=n} F^(k)T F^(k)) unfold_n(G)^T
 *   Num_G = X x_1 F^(1)T ... x_d F^(d)T,  Den_G = G x_1 F^(1)T F^(1) ...
 * (the unfoldings follow Eq. unfolding:property).
 *
 *  X          device, dims[0] x ... x dims[d-1], entries >= 0 and finite
 *  d          3 or 4. d = 4 runs the same sweep on the d-way mode-product
 *             machinery of the differentiation form (two passes over X per
 *             sweep, the FP32 passes on the TF32x3 tensor-core kernel with X
 *             viewed as dims[0] x dims[1]*dims[2] x dims[3]); it has no
 *             NNC_BF16_REFINE form (UNSUPPORTED)
 *  dims, m    host arrays of d entries; 1 <= m[n] <= 64, dims[n] >= 1
 *  F          host array of d device pointers: initial F^(n) (> 0) in,
 *             fitted F^(n) out
 *  G          device: initial core (> 0) in, fitted core out
 *  rel_err_trace  device array of opts->iters doubles, or NULL: relative
 *             error ||X - X_hat||_F / ||X||_F (Sec. 4.1) after each sweep,
 *             from the FP64 identity ||X||^2 - 2<Num_G, G> + <G, Den_G(G)>
 *  rel_err    host, or NULL: final relative error from one explicit FP64
 *             pass over X (as recon_residual)
 * Errors: INVALID_ARG, NEGATIVE_INPUT, NONFINITE (X holds a NaN or an
 * infinity, checked before any sweep; or the FP64 residual terms of some
 * sweep were not finite, i.e. the fit overflowed or produced a NaN: every
 * sweep's trace entry is checked on the device and the call reports the first
 * bad sweep in nnc_last_error_detail), UNSUPPORTED (NNC_BF16_REFINE,
 * exact_every or refine_tol with d = 4), CUDA, ALLOC, TIMEOUT.
 */
int ntd_fit(const void* X, int d, const int64_t* dims, const int* m, int precision,
            const nnc_opts* opts, void* const* F, void* G, double* rel_err_trace,
            double* rel_err, void* stream);

/* One nnTD problem of a batch (see ntd_fit for the meaning of each field). */
typedef struct {
  const void* X;        /* device, C order, d = 3 or 4 modes dims[0..d-1]          */
  int d;
  int64_t dims[4];
  int m[4];
  void* F[4];           /* device F^(n), dims[n] x m[n]: initial in, fitted out     */
  void* G;              /* device core, m[0] x ... x m[d-1]: initial in, fitted out */
  double* trace;        /* device, opts->iters doubles, or NULL                     */
} ntd_job;

/*
 * ntd_fit_batched - many independent ntd_fit problems of uneven shapes (the
 * batching form: several tensors, several multiranks or restarts). The jobs
 * are spread over `concurrency` host workers (0: 8, at most 32), each with a
 * CUDA stream of its own that first waits for the work already queued on
 * `stream`, so small problems overlap on the GPU; every job runs exactly the
 * kernels of ntd_fit and gives the same bits. Returns when all jobs are done.
 * Each worker drives three streams (the sweep graph has side branches): above
 * two workers, start the process with CUDA_DEVICE_MAX_CONNECTIONS raised (e.g.
 * to 32), or the streams share the 8 default hardware queues and partly
 * serialise.
 *
 *  jobs       host array of n_jobs descriptors
 *  rel_errs   host, n_jobs doubles (NaN for a failed job), or NULL
 *  statuses   host, n_jobs status codes, or NULL
 * Errors: the first failing job's status (nnc_last_error_detail names it);
 * INVALID_ARG for bad arguments of the call itself.
 */
int ntd_fit_batched(int n_jobs, const ntd_job* jobs, int precision, const nnc_opts* opts,
                    int concurrency, double* rel_errs, int* statuses, void* stream);

/*
 * Batched fits of small problems, one thread block per problem: many random
 * starts of Alg. 1 and Alg. 2 on a small tensor (the multirank study of
 * Sec. 4.3 on Ex. "equal": a 4 x 4 x 4 tensor, several multiranks, many
 * starts) and many small tensors (the 1000 planted 40 x 40 x 40 tensors of
 * Sec. 4.3). When every job's data fits in shared memory it all goes there;
 * otherwise (ntd_fit_small_batched) the whole batch keeps X in global memory
 * and reads it twice per sweep like ntd_fit, with the factors, core and pass
 * results in shared memory (then m[n] <= 16); lifted_rel_err_batched always
 * streams X. Pointers inside the descriptors are device pointers; the
 * descriptor arrays are host arrays copied by the call. rel_errs: device,
 * n_jobs doubles (final relative error of each job), or NULL. Same update
 * rules as ntd_fit and nmf_fit. Errors: INVALID_ARG, UNSUPPORTED (a job too
 * large for one block), CUDA, ALLOC. No host synchronisation.
 */
typedef struct {
  const void* X;        /* dims[0] x dims[1] x dims[2], C order                    */
  int dims[3];
  int m[3];             /* 1 <= m[n] <= 32                                        */
  void* F[3];           /* dims[n] x m[n]: initial in, fitted out                  */
  void* G;              /* m[0] x m[1] x m[2]: initial in, fitted out              */
} ntd_small_job;

typedef struct {
  const void* A;        /* N x r (read only)                                       */
  int N, r, m;
  void* F;              /* N x m: initial in, fitted out                           */
  void* B;              /* m x r: initial in, fitted out                           */
} nmf_job;

typedef struct {
  const void* X;        /* dims[0] x dims[1] x dims[2]                             */
  int dims[3];
  int m[3];
  int r;
  const void* F[3];     /* dims[n] x m[n]                                          */
  const void* B[3];     /* m[n] x r                                                */
} lifted_job;

/* nnTD (Alg. 1, step 1) of every job, opts->iters sweeps; rel_errs gets
 * ||X - G x_k F^(k)|| / ||X||. */
int ntd_fit_small_batched(int n_jobs, const ntd_small_job* jobs, int precision,
                          const nnc_opts* opts, double* rel_errs, void* stream);
/* NMF A ~ F B (Alg. 2, step 2) of every job; rel_errs gets ||A - F B|| / ||A||. */
int nmf_fit_batched(int n_jobs, const nmf_job* jobs, int precision, const nnc_opts* opts,
                    double* rel_errs, void* stream);
/* rel_errs[j] = ||X - I x_k F^(k) B^(k)|| / ||X|| of every job (the
 * nnCANDELINC objective, Eq. nnCANDELINC, of a fitted pair). */
int lifted_rel_err_batched(int n_jobs, const lifted_job* jobs, int precision, double* rel_errs,
                           void* stream);

/*
 * nncp_core_fit - nonnegative CP decomposition G ~ I x_1 B^(1) ... x_d B^(d)
 * of a core (Alg. 1, step 2; model Eq. npd). opts->iters sweeps over
 * B^(1), ..., B^(d) of
 *   B^(n) <- max(B^(n) * (unfold_n(G) KR_{k!=n} B^(k)) / max(B^(n) V_n, eps), 0),
 *   V_n = Hadamard product over k != n of B^(k)T B^(k),
 * with the Khatri-Rao rows ordered like the unfolding columns (Sec. 3.1).
 *
 *  G          device core, m[0] x ... x m[d-1], entries >= 0
 *  d          3 or 4;  1 <= m[n] <= 64;  1 <= r <= 32
 *  precision  NNC_FP64 or NNC_FP32 (NNC_BF16_REFINE is taken as NNC_FP32)
 *  B          host array of d device pointers: initial B^(n) (> 0) in,
 *             fitted B^(n) out
 *  rel_err    host, or NULL: final ||G - I x_n B^(n)||_F / ||G||_F (FP64 sums)
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, ALLOC; NONFINITE when rel_err is
 * asked for and is not finite (a NaN or an overflow in the fit).
 */
int nncp_core_fit(const void* G, int d, const int* m, int r, int precision, const nnc_opts* opts,
                  void* const* B, double* rel_err, void* stream);

/* One independent core fit of nncp_core_fit_batched. */
typedef struct {
  const void* G;  /* device core, m[0] x ... x m[d-1]             */
  int d;          /* 3 or 4                                        */
  int m[4];       /* core dimensions, 1 <= m[n] <= 64              */
  int r;          /* CP rank, 1 <= r <= 32                         */
  void* B[4];     /* device B^(n), m[n] x r: initial in, fitted out */
} nncp_job;

/*
 * nncp_core_fit_batched - many independent nncp_core_fit problems (uneven
 * shapes and ranks: restarts, candidate ranks, several tensors) in one
 * launch, one thread block per job. Same update rule and options as
 * nncp_core_fit. A batch holding a large tensor (16384 entries or more, such
 * as X itself in Alg. 2, e.g. 40 x 40 x 40) runs with the tensors read twice
 * per sweep from global memory when every job is 3-way with r <= 16 and its
 * arrays fit one block; when, besides, each job's slabs fit a block and one
 * cluster of eight blocks per job fits on the GPU at once (a few large fits,
 * such as the 32 x 32 x 32 core of Alg. 1), each job runs on such a cluster,
 * its blocks sharing the sweep through distributed shared memory. A batch
 * whose state does not fit shared memory and that neither form can take is
 * UNSUPPORTED. The same holds for nncp_core_fit.
 *
 *  jobs       host array of n_jobs descriptors (copied by the call)
 *  rel_errs   device array of n_jobs doubles, or NULL: final relative error
 *             of each job
 *  statuses   device array of n_jobs ints, or NULL: the status of each fit,
 *             written by the fit's own block when the launch ends:
 *               NNC_OK;
 *               NNC_ERR_NONFINITE   a NaN or an infinity in the fitted B^(n)
 *                                   or in the FP64 residual sums (e.g. a NaN
 *                                   or an overflow in the job's core);
 *               NNC_ERR_INVALID_ARG the descriptor is bad (d, m, r or a NULL
 *                                   pointer); the job is skipped, its arrays
 *                                   are not touched.
 *             No wait in these kernels is bounded by time (they have none),
 *             so a fit never reports NNC_ERR_TIMEOUT.
 * Errors: INVALID_ARG (bad options; with statuses NULL also any bad job
 * descriptor; with statuses given a bad descriptor only marks its job and the
 * other jobs run), UNSUPPORTED (see above), CUDA, ALLOC. No host
 * synchronisation.
 */
int nncp_core_fit_batched(int n_jobs, const nncp_job* jobs, int precision, const nnc_opts* opts,
                          double* rel_errs, int* statuses, void* stream);

/*
 * nncp_core_fit_batched_noalloc - nncp_core_fit_batched for callers that must
 * not allocate device memory. The paper has no counterpart: this is a service
 * of the library, not a step of the method.
 *
 * Who needs it: a host runtime that owns all device memory through its own
 * pool and forbids a library to allocate behind its back; a latency-critical
 * loop where an allocation may stall, or fail when the GPU's memory is nearly
 * all handed out. The allocating call takes its job table from cudaMallocAsync;
 * this one keeps the table in a fixed array inside the library's device memory
 * (4096 descriptors, 256 KiB, held on every GPU that loads the library until
 * the process exits) and calls no allocator at all.
 *
 * Arguments, results, statuses and errors are those of nncp_core_fit_batched,
 * and every batch it accepts runs the same one-pass kernel with the same sums,
 * except:
 *  - batches that nncp_core_fit_batched sends to its two-pass kernel (a tensor
 *    of 16384 entries or more, such as X in Alg. 2, or state beyond one block:
 *    see above) are refused with NNC_ERR_UNSUPPORTED, because that kernel's
 *    table is allocated; nnc_last_error_detail says so;
 *  - n_jobs > 4096 is rejected with NNC_ERR_INVALID_ARG (nnc_last_error_detail
 *    says so);
 *  - it never times block sizes: it reuses the size an earlier allocating call
 *    of the same shape class chose (the results are the same bits either way);
 *  - the first call on a device looks up the table's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture;
 *  - every call writes the one shared table: calls whose work may overlap on
 *    the GPU (other streams, other threads) race and must be ordered by the
 *    caller;
 *  - the descriptors are copied with cudaMemcpyAsync on `stream`; from
 *    pageable host memory the copy is done when the call returns, from
 *    page-locked memory keep `jobs` unchanged until `stream` has reached it.
 */
int nncp_core_fit_batched_noalloc(int n_jobs, const nncp_job* jobs, int precision,
                                  const nnc_opts* opts, double* rel_errs, int* statuses,
                                  void* stream);

/*
 * nnc_mode_product - the n-mode product of Appendix A (Def. of n-mode
 * multiplication) with A = F^T, for a 3-way X:
 *   Y[.., q, ..] = sum_l X[.., l, ..] F[l, q]     (mode `mode` of size Q in Y)
 * These are the contractions of the two passes over X of every nnTD sweep
 * (mode 2 = X x_3 F^(3)T, mode 0 = X x_1 F^(1)T), exposed on their own.
 *
 *  X          device, dims[0] x dims[1] x dims[2]
 *  mode       0, 1 or 2 (index 0 is mode 1 of the paper)
 *  F          device, dims[mode] x Q row-major; 1 <= Q <= 64
 *  out        device, dims with dims[mode] replaced by Q, C order
 *  precision  NNC_FP64 (double), NNC_FP32_SIMT (float): SIMT kernels.
 *             NNC_FP32 (float): TF32x3 tensor cores: tcgen05 passes for
 *             modes 0 and 2, mma.sync column products for mode 1 when
 *             N3 % 4 == 0 and Q <= 32; SIMT otherwise (N3 % 4 != 0, or
 *             mode 1 with Q > 32).
 *             NNC_BF16_REFINE (float X, F, out): tensor cores on BF16 copies
 *             of X and F (X scaled per mode-1 slice by a power of two, which
 *             changes no rounding) with FP32 accumulation; modes 0 and 2 only.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA, ALLOC, TIMEOUT.
 */
int nnc_mode_product(const void* X, int d, const int64_t* dims, int mode, const void* F, int Q,
                     int precision, void* out, void* stream);

/*
 * candelinc_lift - A^(n) = F^(n) B^(n) for every mode: the CPD of the core
 * substituted into the Tucker model (proof of Lemma "rank and min exists",
 * Sec. 2.1), giving the CP factors of the nnCANDELINC model.
 *
 *  F, B, A    host arrays of d device pointers (A^(n) is dims[n] x r)
 * Errors: INVALID_ARG, CUDA.
 */
int candelinc_lift(int d, const int64_t* dims, const int* m, int r, int precision,
                   const void* const* F, const void* const* B, void* const* A, void* stream);

/*
 * candelinc_lifted_grad - the adjoint of the nnCANDELINC objective with the
 * CPD of the core substituted (Eq. nnCANDELINC, Sec. 4; the substitution
 * A^(n) = F^(n) B^(n) of the proof of Lemma "rank and min exists"):
 *   L = 1/2 ||X - I x_n F^(n) B^(n)||_F^2,
 *   dL/dA^(n) = A^(n) V_n - unfold_n(X x_{k!=n} F^(k)T) KR_{k!=n}(B^(k)),
 *   V_n = Hadamard_{k!=n} A^(k)T A^(k),
 *   dL/dF^(n) = dL/dA^(n) B^(n)T,   dL/dB^(n) = F^(n)T dL/dA^(n).
 * Reads X twice (X x_d F^(d)T and X x_1 F^(1)T; once when only the loss is
 * asked for).
 *
 *  X          device, C order, d = 3 or 4 modes dims[0..d-1]
 *  m, r       m[n] <= 64, 1 <= r <= 64
 *  F, B       host arrays of d device pointers: F^(n) dims[n] x m[n],
 *             B^(n) m[n] x r, row-major (read only)
 *  gF, gB     host arrays of d device pointers shaped like F and B (written),
 *             or both NULL for the loss alone
 *  loss       host, L with FP64 accumulation (may be NULL when gF is given)
 *  precision  NNC_FP64 (double); NNC_FP32 (float, TF32x3 tensor-core passes
 *             where the shape allows, else SIMT); NNC_FP32_SIMT (float)
 * Errors: INVALID_ARG, NONFINITE (X), UNSUPPORTED (NNC_BF16_REFINE), CUDA,
 * ALLOC, TIMEOUT.
 */
int candelinc_lifted_grad(const void* X, int d, const int64_t* dims, const int* m, int r,
                          int precision, const void* const* F, const void* const* B,
                          void* const* gF, void* const* gB, double* loss, void* stream);

/*
 * candelinc_pg_fit - `steps` block-coordinate projected-gradient steps on the
 * same L, in place on F and B. The paper gives no first-order method for Eq.
 * nnCANDELINC; the reading taken: for n = 1..d,
 *   F^(n) <- max(F^(n) - dL/dF^(n) / L_F, 0),  L_F = lmax(B^(n) V_n B^(n)T),
 *   B^(n) <- max(B^(n) - dL/dB^(n) / L_B, 0),  L_B = lmax(F^(n)T F^(n)) lmax(V_n),
 * the B gradient taken after the F update, lmax from 30 FP64 power iterations
 * from the all-ones vector (Rayleigh quotient). Each block problem is a convex
 * quadratic, so no step increases L. Two passes over X per step.
 *
 *  trace      device, `steps` doubles (L after each step), or NULL
 *  loss       host, L after the last step (NaN for steps = 0), or NULL
 *  (other arguments as candelinc_lifted_grad; F and B are read and written)
 * Errors: as candelinc_lifted_grad; NONFINITE also when the loss of some
 * step was not finite (an overflow or a NaN during the fit).
 */
int candelinc_pg_fit(const void* X, int d, const int64_t* dims, const int* m, int r,
                     int precision, int steps, void* const* F, void* const* B, double* trace,
                     double* loss, void* stream);

/*
 * nncp_tensor_fit - nnCPD of X itself, the first step of Alg. 2 (Sec. 4.1):
 * `opts->iters` Gauss-Seidel MU sweeps on the CP factors,
 *   A^(n) <- max(A^(n) .* MT_n / max(A^(n) V_n, eps), 0),
 *   MT_n = unfold_n(X) KR_{k!=n}(A^(k)),  V_n = Hadamard_{k!=n} A^(k)T A^(k)
 * (the rule of nncp_core_fit with X in place of the core), two passes over X
 * per sweep.
 *
 *  X          device, C order, d = 3 or 4 modes dims[0..d-1]
 *  A          host array of d device pointers, A^(n) dims[n] x r (1 <= r <= 64),
 *             initial values on entry, result on exit
 *  trace      device, opts->iters doubles: ||X - I x_k A^(k)||_F / ||X||_F after
 *             each sweep (FP64 identity; with opts->exact_every = k > 0 every
 *             k-th entry and the last from one explicit FP64 pass over X), or
 *             NULL
 *  rel_err    host, the final relative error from one explicit FP64 pass over
 *             X (NaN for 0 sweeps), or NULL
 *  precision  NNC_FP64, NNC_FP32 (TF32x3 tensor-core passes), NNC_FP32_SIMT
 * Errors: INVALID_ARG, NONFINITE (X, or a sweep whose FP64 residual terms
 * were not finite), UNSUPPORTED, CUDA, ALLOC, TIMEOUT.
 */
int nncp_tensor_fit(const void* X, int d, const int64_t* dims, int r, int precision,
                    const nnc_opts* opts, void* const* A, double* trace, double* rel_err,
                    void* stream);

/*
 * nmf_fit - the NMF A ~ F B of one CP factor, the second step of Alg. 2 (Sec.
 * 4.1): `opts->iters` MU iterations (Lee-Seung),
 *   F <- max(F .* (A B^T) / max(F B B^T, eps), 0),
 *   B <- max(B .* (F^T A) / max(F^T F B, eps), 0).
 *
 *  A          device, N x r row-major (read only)
 *  F, B       device, N x m and m x r row-major, initial values in, result out
 *  trace      device, opts->iters doubles: ||A - F B||_F / ||A||_F, or NULL
 *  rel_err    host, the last value (NaN for 0 iterations), or NULL
 *  precision  NNC_FP64 (double) or NNC_FP32 / NNC_FP32_SIMT (float)
 * Errors: INVALID_ARG, NONFINITE (an iteration's residual was not finite),
 * UNSUPPORTED, CUDA, ALLOC.
 */
int nmf_fit(const void* A, int64_t N, int r, int m, int precision, const nnc_opts* opts, void* F,
            void* B, double* trace, double* rel_err, void* stream);

/*
 * candelinc_alg2 - Alg. 2 (Sec. 4.1): A = nnCPD(X, r) by nncp_tensor_fit
 * (cp_opts), then F^(n), B^(n) = NMF(A^(n), m[n]) by nmf_fit (nmf_opts) for
 * every mode. A, F, B hold the initial values on entry. cp_rel_err (host) gets
 * the CP fit, nmf_rel_errs (host, d doubles) the NMF fits; either may be NULL.
 * Errors: as nncp_tensor_fit and nmf_fit.
 */
int candelinc_alg2(const void* X, int d, const int64_t* dims, const int* m, int r, int precision,
                   const nnc_opts* cp_opts, const nnc_opts* nmf_opts, void* const* A,
                   void* const* F, void* const* B, double* cp_rel_err, double* nmf_rel_errs,
                   void* stream);

/*
 * recon_residual - ||X - X_hat||_F and ||X||_F in one pass over X with FP64
 * accumulation (the relative error of Sec. 4.1 is their ratio).
 *
 *  model 0: Tucker X_hat = G x_1 F^(1) ... (factors = F, dims[n] x m[n])
 *  model 1: CP     X_hat = I x_1 A^(1) ... (factors = A, dims[n] x r; G and m
 *           unused)
 *  resid_norm, x_norm  host
 *  d          3 or 4
 * Errors: INVALID_ARG, CUDA, ALLOC.
 */
int recon_residual(const void* X, int d, const int64_t* dims, int precision, int model,
                   const int* m, int r, const void* const* factors, const void* G,
                   double* resid_norm, double* x_norm, void* stream);

/*
 * Tracing aid: CUDA-event timing of the two passes over X of nnTD sweeps,
 * the kernels that dominate ntd_fit. While enabled, ntd_fit (d = 3) records
 * an event pair around each pass of every 16th sweep (the 16th, the 32nd, ...) on the
 * stream that launches it; the pairs are read (synchronising on them) by
 * nnc_profile_read, not inside ntd_fit.
 * Kinds:
 *   0  X x_3 F^(3)T, SIMT passes (NNC_FP64, NNC_FP32_SIMT)
 *   1  X x_1 F^(1)T, SIMT passes
 *   2  X x_3 F^(3)T, BF16 tensor-core passes
 *   3  X x_1 F^(1)T, BF16 tensor-core passes
 *   4  X x_3 F^(3)T, TF32x3 tensor-core passes (NNC_FP32, refinement sweeps)
 *   5  X x_1 F^(1)T, TF32x3 tensor-core passes
 * nnc_profile_enable(on) switches it and clears the totals; nnc_profile_read
 * returns the number of timed launches and their total milliseconds of a
 * kind. Meant for one thread of control: concurrent ntd_fit calls while it is
 * enabled share one event pool and give meaningless totals.
 */
int nnc_profile_enable(int on);
int nnc_profile_read(int kind, long long* launches, double* total_ms);

/* Running count of the CUDA kernels this library has launched in this
 * process (a kernel node of a replayed graph counts once per replay). */
long long nnc_kernel_launches(void);

/*
 * Launch-shape autotuner of the batched one-block-per-job fits
 * (nncp_core_fit[_batched], ntd_fit_small_batched, nmf_fit_batched). On (the
 * default), the first call of a new shape class (kernel, element size, size
 * classes of the largest job and of the job count; per device) spends its
 * first sweeps on trial launches at 32, 64, 128 and 256 threads per block,
 * timed with events (one host wait in that call), and runs the remaining
 * sweeps, and every later call of the class, at the fastest. The results are
 * the same bits whatever the choice: the sweeps of a fit may be split over
 * launches and no sum depends on the block size. Off: 256 threads, no
 * timing. nncp_core_fit_batched_noalloc uses a cached choice but never
 * times. nnc_autotune_enable returns the previous setting. Calls made while
 * the stream is being captured into a graph never time either.
 */
int nnc_autotune_enable(int on);

/*
 * Failure-detection self-test (not a step of the method). Every wait of the
 * tensor-core pass kernel on an mbarrier is bounded: past its limit the role
 * that waits flags the CTA as failed, the others stop, and the call returns
 * NNC_ERR_TIMEOUT instead of hanging. This runs that same wait once, in a
 * one-CTA kernel, on a barrier that expects one arrival and gets none (no
 * copy or MMA is in flight), with a limit of `cycles` SM clocks (a few
 * million: about a millisecond). Returns NNC_ERR_TIMEOUT when the wait gave
 * up, as it must, and NNC_OK if it returned; the CUDA context stays usable.
 */
int nnc_wait_selftest(long long cycles, void* stream);

/*
 * Failure-injection hook for tests (not a step of the method; off by
 * default). Arms the nth scratch allocation from now (nth >= 1; 0 disarms) to
 * fail on the host as if cudaMallocAsync had returned an error, without
 * calling the allocator: the call that makes it returns NNC_ERR_ALLOC, releases
 * the scratch it already holds, and leaves the CUDA context usable. Shared by
 * every thread of the process. Returns the previous countdown.
 */
int nnc_debug_fail_alloc(int nth);

/* The sweep index (0-based) at which the last NNC_BF16_REFINE ntd_fit call of
 * this thread began its FP32 refinement sweeps (iters when it ran none), or -1
 * when this thread has made no such call. */
int nnc_last_refine_sweep(void);

/* Static string naming a status code. */
const char* nnc_status_string(int status);

/* Text of the last CUDA error seen by this thread's calls (empty if none). */
const char* nnc_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* NNCANDELINC_H */
