// nnTD of a 3-way tensor (Alg. 1, step 1) on the GPU: the sweep loop.
//
// One sweep updates F^(1), F^(2), F^(3) and then G (Gauss-Seidel), each by the
// multiplicative rule theta <- max(theta * Num / max(Den, eps), 0) whose
// Den - Num is the gradient of 1/2 ||X - G x_k F^(k)||^2 (Eq. unfolding:property):
//
//   pass 1   P3 = X x_3 F3^T                          (first read of X)
//   upd 1    Num1 = unfold_1(P3 x_2 F2^T) unfold_1(G)^T,  Den1 = F1 H1
//   hmat 2   H2 = unfold_2(G x_1 S1 x_3 S3) unfold_2(G)^T
//   upd 2    Num2 from P3 x_1 F1^T (new F1),  Den2 = F2 H2  (numerator beside H2)
//   hmat 3   H3 from W3 = G x_1 S1 x_2 S2 (W3 kept)
//   pass 2   P1 = X x_1 F1^T (new F1), rows (k, j)     (second read of X)
//   upd 3    Y3 = P1 x_2 F2^T (new F2);  Num3 = unfold_3(Y3) unfold_3(G)^T;  Den3 = F3 H3
//            (numerator beside H3)
//   core     M = Y3 x_3 F3^T = X x_1 F1^T x_2 F2^T x_3 F3^T;
//            G <- MU(G, M, W3 x_3 S3); trace; next H1       (core_a, core_b)
// with S_k = F_k^T F_k. The kernels are in sweep.cu; the passes are SIMT mode
// products (ttm.cu) or, on the BF16 path, tensor-core mode products from a
// BF16 copy of X (tc_ttm.cu). Two reads of X per sweep is the minimum under
// the Gauss-Seidel order: pass 2 needs the F^(1) that pass 1 leads to.
//
// The sweep is captured as a CUDA graph on a private stream (several sweeps to
// a graph) and replayed; the trace slot advances through a device counter. NNC_FP32 runs the passes
// as FP32-accurate TF32x3 tensor-core products; NNC_BF16_REFINE replays the
// BF16 tensor-core sweep for iters - refine_iters sweeps and then the TF32x3
// sweep for the rest; NNC_FP32_SIMT and NNC_FP64 use the SIMT passes.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "ntd.cuh"
#include "profile.cuh"
#include "residual.cuh"
#include "sweep.cuh"
#include "tc_ttm.cuh"

namespace nnc {

namespace {

template <typename T>
struct NtdState {
  int64_t N[3];
  int m[3];
  // P3 rows (i, j) x m3; P1 rows (k, j) x m1 (SIMT passes: P1s, laid out
  // (m1, N2, N3), is the pass result that P1 is copied from)
  T *P3, *P1, *P1s, *Y3, *M, *W1, *W3, *G2, *G3, *H[3], *S[3];
  T *num2, *num3;  // numerators of the split mode-2 and mode-3 updates
  T* Yb;           // Y_r of the mode-1 and mode-2 tensor-core updates (UpdArgs::ybuf)
  // Shares of Y1[i] = F2^T P3[i] and of Y3[k] = P1[k]^T F2 from the
  // tensor-core passes (y_nh = N2 / 128 per slab; NULL: the update kernel forms them)
  T* Y1p;
  T* Y3p;
  int y_nh;
  double *stats_part, *stats, *trace_dummy, *resid2, *dots;
  int* counter;
  int* done;
  int* gate;
};

template <typename T>
int pass_x3(const T* X, const NtdState<T>& b, const T* F3, const T* F2, const tc::TcPlan* tcp,
            cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (tcp) {
      if (b.Y1p && tcp->y1_fusable(b.m[1]))
        return tcp->pass3(F3, b.P3, s, /*convert=*/false, F2, b.m[1], b.Y1p);
      return tcp->pass3(F3, b.P3, s, /*convert=*/false);
    }
  }
  // No split buffer: the passes fill the GPU without splitting the contraction.
  NNC_CUDA_TRY(launch_ttm<T>(X, b.N[0] * b.N[1], (int)b.N[2], 1, F3, b.m[2], 1, b.m[2], b.P3,
                             nullptr, 0, s));
  return NNC_OK;
}

template <typename T>
int pass_x1(const T* X, const NtdState<T>& b, const T* F1, const T* F2, const tc::TcPlan* tcp,
            cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (tcp) {
      if (F2) return tcp->pass1(F1, b.P1, s, /*convert=*/false, F2, b.m[1], b.Y3p);
      return tcp->pass1(F1, b.P1, s, /*convert=*/false);
    }
  }
  NNC_CUDA_TRY(launch_ttm<T>(X, 1, (int)b.N[0], b.N[1] * b.N[2], F1, b.m[0], 1, b.m[0], b.P1s,
                             nullptr, 0, s));
  return launch_p1_rows<T>(b.P1s, b.m[0], b.N[1], b.N[2], b.P1, s);
}

// The tensor-core form of the factor updates' GEMMs (UpdArgs::tc): TF32
// beside BF16 passes, whose rounding of X dominates; split TF32 (FP32-accurate)
// beside TF32x3 passes; none on the SIMT path.
inline int upd_tc(const tc::TcPlan* tcp) {
  return tcp ? (tcp->kind == tc::kKindBf16 ? 1 : 3) : 0;
}

// The core update of a sweep (G, the next H1, the trace entry).
template <typename T>
int launch_sweep_core(T* const* F, T* G, NtdState<T>& b, double eps, double* trace,
                      int trace_stride, const tc::TcPlan* tcp, cudaStream_t s) {
  CoreArgs<T> c{};
  c.G = G;  c.G2 = b.G2;  c.G3 = b.G3;  c.Y3 = b.Y3;  c.Mout = b.M;  c.W3 = b.W3;
  c.S1 = b.S[0];  c.S2 = b.S[1];  c.F3 = F[2];  c.n3 = b.N[2];  c.S3_out = b.S[2];
  c.W1 = b.W1;  c.H1 = b.H[0];  c.dots = b.dots;  c.done = b.done;  c.x2 = b.stats;
  c.trace = trace;  c.trace_stride = trace_stride;  c.counter = b.counter;  c.gate = b.gate;
  c.m1 = b.m[0];  c.m2 = b.m[1];  c.m3 = b.m[2];  c.eps = eps;
  c.tc = upd_tc(tcp);
  c.err = tcp ? tcp->err : nullptr;
  return launch_core<T>(c, s);
}

// Side streams and fork/join events of the concurrent branches of a sweep.
struct Branch {
  cudaStream_t s2 = nullptr, s3 = nullptr;
  cudaEvent_t fork[2] = {}, join[2] = {}, mid[2] = {};
};

// One sweep without its core update, which the next sweep runs (or the caller
// after the last one). Beside the passes, on side streams:
//   pass 1 (X x_3 F3^T)  beside  the previous sweep's core update (G, H1, trace):
//                        the pass needs only F3;
//   pass 2 (X x_1 F1^T)  beside  H3 (and, when it forms the mode-3 shares and so
//                        waits for the new F2, nothing else; otherwise beside
//                        H2, the mode-2 numerator and the MU step on F2 too).
// The passes leave SMs free when that costs them nothing (tc_ttm.cu), and the
// small kernels run there.
template <typename T>
int sweep3(const T* X, T* const* F, T* G, NtdState<T>& b, double eps, double* trace,
           int trace_stride, const PassEvents* ev, const tc::TcPlan* tcp, bool prev_core,
           const Branch& br, cudaStream_t s) {
  const int64_t N1 = b.N[0], N2 = b.N[1], N3 = b.N[2];
  const int m1 = b.m[0], m2 = b.m[1], m3 = b.m[2];

  // ---- previous core beside pass 1; mode 1 -----------------------------------
  if (prev_core) {
    NNC_CUDA_TRY(cudaEventRecord(br.fork[0], s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(br.s2, br.fork[0], 0));
    NNC_TRY(launch_sweep_core<T>(F, G, b, eps, trace, trace_stride, tcp, br.s2));
    NNC_CUDA_TRY(cudaEventRecord(br.join[0], br.s2));
  }
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->start[0], s, cudaEventRecordExternal));
  NNC_TRY(pass_x3<T>(X, b, F[2], F[1], tcp, s));
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->stop[0], s, cudaEventRecordExternal));
  if (prev_core) NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.join[0], 0));
  {
    UpdArgs<T> u{};
    u.P = b.P3;  u.prow = N2 * m3;  u.pstride = m3;  // P3[i, j, c]
    u.Fc = F[1]; u.len = (int)N2;   u.mu = m2;  u.mc = m3;
    u.Gn = G;    // rows a of G are (b, c)-contiguous
    if (tcp && b.Y1p && tcp->y1_fusable(m2)) {  // the pass formed Y1's shares
      u.Ypart = b.Y1p;
      u.nparts = b.y_nh;
    }
    u.F = F[0];  u.nrows = N1;  u.mv = m1;  u.H = b.H[0];  u.eps = eps;
    u.tc = upd_tc(tcp);
    u.err = tcp ? tcp->err : nullptr;
    u.ybuf = b.Yb;
    if constexpr (std::is_same<T, float>::value) {
      if (tcp) {
        u.bt = tcp->Bt1;
        u.bhi = tcp->B1hi;
        u.blo = tcp->B1lo;
        u.bt_ld = tcp->kp1;
        u.bt_scale = tcp->kind == tc::kKindBf16 ? tcp->scale : nullptr;
      }
    }
    NNC_TRY(launch_upd12<T>(u, s));
  }
  // ---- modes 2 and 3 --------------------------------------------------------
  // The numerators do not need H_n, so the mode-2 update is split in two: the
  // GEMM and the numerator (launch_upd12, num_only) run beside the kernel
  // forming H2, and a row-wise MU step follows; in the tensor-core form the
  // GEMM runs beside H2 and one kernel forms the numerators and takes the MU
  // step.
  //   s2:  H2 ................ MU on F2 | H3 (S2 of the new F2)
  //   s3:  Num2 (P3, new F1) --^
  // When pass 2 can also form the shares of Y3[k] = P1[k]^T F2 (TF32x3 with
  // N2 % 128 == 0, m <= 32), it waits for the new F2 and the mode-3 update
  // only adds the shares; H3 runs beside the pass:
  //   s:   pass 2 (new F1, new F2) -- mode 3 (shares, H3)
  // Otherwise pass 2 runs beside the mode-2 branch and the mode-3 numerator
  // beside H3:
  //   s:   pass 2 (new F1) ....... Num3 (P1, new F2) -- MU on F3
  bool y3f = false;
  if constexpr (std::is_same<T, float>::value) y3f = tcp && b.Y3p && tcp->y3_fusable(m2);
  NNC_CUDA_TRY(cudaEventRecord(br.fork[1], s));
  NNC_CUDA_TRY(cudaStreamWaitEvent(br.s2, br.fork[1], 0));
  NNC_CUDA_TRY(cudaStreamWaitEvent(br.s3, br.fork[1], 0));
  {  // H2 from S1 = F1^T F1 (new F1) and S3
    HArgs<T> h{};
    h.Gn = b.G2;  h.mp = m2;  h.mu = m1;  h.mv = m3;
    h.fu = F[0];  h.nu = N1;  h.su_out = b.S[0];
    h.sv = b.S[2];
    h.H = b.H[1];
    h.tc = upd_tc(tcp);
    h.err = tcp ? tcp->err : nullptr;
    NNC_TRY(launch_hmat<T>(h, br.s2));
  }
  UpdArgs<T> u2{};
  u2.P = b.P3;  u2.prow = m3;  u2.pstride = N2 * m3;  // row j, contraction over i
  u2.Fc = F[0]; u2.len = (int)N1;  u2.mu = m1;  u2.mc = m3;
  u2.Gn = b.G2;  // rows b of G2 are (a, c)-contiguous
  u2.F = F[1];  u2.nrows = N2;  u2.mv = m2;  u2.H = b.H[1];  u2.eps = eps;
  u2.num = b.num2;
  u2.num_only = 1;
  u2.tc = upd_tc(tcp);
  u2.err = tcp ? tcp->err : nullptr;
  u2.ybuf = b.Yb;
  bool tc2 = false;
  if constexpr (std::is_same<T, float>::value) tc2 = upd_tc_form(u2);
  if (tc2) {
    // Tensor-core form: the GEMM beside H2, then numerators and MU in one.
    if constexpr (std::is_same<T, float>::value) {
      NNC_TRY(launch_upd_gemm(u2, br.s3));
      NNC_CUDA_TRY(cudaEventRecord(br.mid[0], br.s3));
      NNC_CUDA_TRY(cudaStreamWaitEvent(br.s2, br.mid[0], 0));
      u2.num_only = 0;
      NNC_TRY(launch_upd_num(u2, br.s2));
    }
  } else {
    NNC_TRY(launch_upd12<T>(u2, br.s3));
    NNC_CUDA_TRY(cudaEventRecord(br.mid[0], br.s3));
    NNC_CUDA_TRY(cudaStreamWaitEvent(br.s2, br.mid[0], 0));
    u2.num_only = 0;
    NNC_TRY(launch_mu_rows<T>(u2, br.s2));
  }
  NNC_CUDA_TRY(cudaEventRecord(br.mid[1], br.s2));  // the new F2
  {  // H3 and W3 = G x_1 S1 x_2 S2, with S2 = F2^T F2 (new F2)
    HArgs<T> h{};
    h.Gn = b.G3;  h.mp = m3;  h.mu = m1;  h.mv = m2;
    h.w_sp = 1;  h.w_su = (int64_t)m2 * m3;  h.w_sv = m3;  // W3 in the layout of G
    h.su = b.S[0];
    h.fv = F[1];  h.nv = N2;  h.sv_out = b.S[1];
    h.H = b.H[2];
    h.Wout = b.W3;
    h.tc = upd_tc(tcp);
    h.err = tcp ? tcp->err : nullptr;
    NNC_TRY(launch_hmat<T>(h, br.s2));
  }
  NNC_CUDA_TRY(cudaEventRecord(br.join[1], br.s2));
  if (y3f) NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.mid[1], 0));
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->start[1], s, cudaEventRecordExternal));
  NNC_TRY(pass_x1<T>(X, b, F[0], y3f ? F[1] : nullptr, tcp, s));
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->stop[1], s, cudaEventRecordExternal));
  UpdArgs<T> u3{};
  u3.P = b.P1;  u3.prow = N2 * m1;  u3.pstride = m1;  // P1[k, j, a]
  u3.Fc = F[1]; u3.len = (int)N2;   u3.mu = m1;  u3.mc = m2;  u3.p_first = 1;
  u3.Gn = b.G3;  // rows c of G3 are (a, b)-contiguous
  u3.Yout = b.Y3;
  u3.F = F[2];  u3.nrows = N3;  u3.mv = m3;  u3.H = b.H[2];  u3.eps = eps;
  u3.gate_out = b.gate;
  u3.tc = upd_tc(tcp);
  u3.err = tcp ? tcp->err : nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (tcp) {
      u3.bt = tcp->Bt3;
      u3.bhi = tcp->B3hi;
      u3.blo = tcp->B3lo;
      u3.bt_ld = tcp->kb3;
    }
  }
  u3.ybuf = b.Y3;  // the tensor-core form's Y3 is the one the core update keeps
  bool tc3 = false;
  if constexpr (std::is_same<T, float>::value) tc3 = !y3f && upd_tc_form(u3);
  if (y3f) {
    u3.Ypart = b.Y3p;
    u3.nparts = b.y_nh;
    NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.join[1], 0));
    NNC_TRY(launch_upd12<T>(u3, s));
  } else if (tc3) {
    if constexpr (std::is_same<T, float>::value) {
      NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.mid[1], 0));
      NNC_TRY(launch_upd_gemm(u3, s));
      NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.join[1], 0));
      NNC_TRY(launch_upd_num(u3, s));
    }
  } else {
    NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.mid[1], 0));
    u3.num = b.num3;
    u3.num_only = 1;
    u3.gate_out = nullptr;
    NNC_TRY(launch_upd12<T>(u3, s));
    NNC_CUDA_TRY(cudaStreamWaitEvent(s, br.join[1], 0));
    u3.num_only = 0;
    u3.gate_out = b.gate;
    NNC_TRY(launch_mu_rows<T>(u3, s));
  }
  return NNC_OK;
}

int count_kernel_nodes(cudaGraph_t graph, long long* n_kernels) {
  size_t n = 0;
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &n));
  long long k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    NNC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++k;
  }
  *n_kernels = k;
  return NNC_OK;
}

// RAII holder of the private streams, graphs and events of one replay loop:
// graph 0 is the sweep, graph 1 its instrumented copy for the profiler.
struct GraphRun {
  cudaStream_t cs = nullptr;
  Branch br;
  cudaGraph_t graph[3] = {};    // one sweep, the instrumented sweep, kSweepsPerGraph sweeps
  cudaGraphExec_t exec[3] = {};
  cudaEvent_t fork = nullptr, join = nullptr;
  ~GraphRun() {
    for (int k = 0; k < 3; ++k) {
      if (exec[k]) cudaGraphExecDestroy(exec[k]);
      if (graph[k]) cudaGraphDestroy(graph[k]);
    }
    for (int k = 0; k < 2; ++k) {
      if (br.fork[k]) cudaEventDestroy(br.fork[k]);
      if (br.join[k]) cudaEventDestroy(br.join[k]);
      if (br.mid[k]) cudaEventDestroy(br.mid[k]);
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (br.s2) cudaStreamDestroy(br.s2);
    if (br.s3) cudaStreamDestroy(br.s3);
    if (cs) cudaStreamDestroy(cs);
  }
};

// While the profiler is on, one sweep in kProfileEvery runs from a second
// capture of the sweep whose passes are bracketed by event-record nodes. Event
// nodes cost the device a few microseconds each, so timing every sweep would
// slow the fit it measures by about a tenth; sampled sweeps are otherwise the
// same kernels on the same data.
constexpr int kProfileEvery = 16;

// Sweeps per replay of the plain graph: consecutive graph launches leave the
// GPU idle for a few microseconds, a kernel boundary inside a graph for less.
// Five keeps every profiled sweep (the last of kProfileEvery) on its own.
constexpr int kSweepsPerGraph = 5;
static_assert(kProfileEvery % kSweepsPerGraph == 1, "sampled sweeps fall between graphs");

template <typename T>
int capture_sweep(const T* X, T* const* F, T* G, NtdState<T>& b, double eps, double* trace,
                  const PassEvents* ev, const tc::TcPlan* tcp, bool prev_core, GraphRun& g,
                  int slot, int nsweeps = 1) {
  NNC_CUDA_TRY(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
  int cap_st = NNC_OK;
  for (int k = 0; k < nsweeps && cap_st == NNC_OK; ++k)
    cap_st = sweep3<T>(X, F, G, b, eps, trace ? trace : b.trace_dummy, trace ? 1 : 0, ev, tcp,
                       prev_core, g.br, g.cs);
  const cudaError_t end_e = cudaStreamEndCapture(g.cs, &g.graph[slot]);
  if (cap_st != NNC_OK) return cap_st;
  NNC_CUDA_TRY(end_e);
  NNC_CUDA_TRY(cudaGraphInstantiate(&g.exec[slot], g.graph[slot], 0));
  return NNC_OK;
}

// Exact checkpoints of the trace and the refinement trigger (nnc_opts
// exact_every, refine_tol). After every exact_every-th sweep of the fit and
// after its last one, the pending core update runs at once and the sweep's
// trace entry is replaced by the relative error of one explicit pass over X
// (FP64 sums, as recon_residual): the residual identity loses accuracy near
// convergence, where ||X - X_hat||^2 is a small difference of large terms
// formed from FP32-accurate (or BF16) quantities.
template <typename T>
struct Checkpoints {
  int every = 0;             // 0: none
  int total = 0;             // sweeps of the whole fit (the last is a checkpoint)
  const T* X = nullptr;
  const int64_t* dims = nullptr;
  const int* m = nullptr;
  const ResidualWork<T>* rw = nullptr;
  // Refinement trigger (fast sweeps only): stop the fast phase at a checkpoint
  // whose relative decrease since the previous checkpoint is below tol times
  // the largest such decrease seen so far in the fit.
  double tol = 0.0;
  double last = -1.0, peak = 0.0;  // host-side history
  bool at(int sweep) const {
    return every > 0 && ((sweep + 1) % every == 0 || sweep + 1 == total);
  }
};

// Captures the sweep on a private stream and replays it `count` times after
// the work already queued on `s`, runs the last sweep's core update, and makes
// `s` wait for all of it. The core update a replay runs first is the previous
// sweep's; in the first replay there is none, and the core kernels see the
// pending flag at 0 and return at once. `first` is the fit's index of the
// first of these sweeps; *done gets the number of sweeps run, fewer than
// `count` when the refinement trigger of `ck` stopped them.
template <typename T>
int run_sweeps(const T* X, T* const* F, T* G, NtdState<T>& b, double eps, double* trace,
               int count, int first, Checkpoints<T>* ck, const tc::TcPlan* tcp, cudaStream_t s,
               int* done) {
  *done = 0;
  if (count <= 0) return NNC_OK;
  GraphRun g;
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.br.s2, cudaStreamNonBlocking));
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.br.s3, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.br.fork[k], cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.br.join[k], cudaEventDisableTiming));
    NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.br.mid[k], cudaEventDisableTiming));
  }
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventRecord(g.fork, s));
  NNC_CUDA_TRY(cudaStreamWaitEvent(g.cs, g.fork, 0));

  NNC_TRY(capture_sweep<T>(X, F, G, b, eps, trace, nullptr, tcp, true, g, 0));
  long long kn[3] = {0, 0, 0};
  NNC_TRY(count_kernel_nodes(g.graph[0], &kn[0]));
  if (count >= kSweepsPerGraph) {
    NNC_TRY(capture_sweep<T>(X, F, G, b, eps, trace, nullptr, tcp, true, g, 2, kSweepsPerGraph));
    NNC_TRY(count_kernel_nodes(g.graph[2], &kn[2]));
  }
  const bool checkpoints = ck && ck->every > 0 && trace;

  // Sampled sweeps: the last of every kProfileEvery (an instrumented copy,
  // captured once the first plain replays are queued, so the device is busy
  // meanwhile).
  PassProfiler prof(tcp ? (tcp->kind == tc::kKindBf16 ? 2 : 4) : 0);
  const int samples = profile_enabled() ? count / kProfileEvery : 0;
  long long kernels = 0;
  int t = 0;
  while (t < count) {
    const bool sampled = samples > 0 && t % kProfileEvery == kProfileEvery - 1;
    // A five-sweep replay must not pass a sampled sweep or a checkpoint (its
    // last sweep may be one).
    bool five = !sampled && g.exec[2] && t + kSweepsPerGraph <= count &&
                (samples == 0 || t % kProfileEvery + kSweepsPerGraph <= kProfileEvery - 1);
    if (five && checkpoints)
      for (int u = t; u < t + kSweepsPerGraph - 1; ++u) five = five && !ck->at(first + u);
    if (five) {
      NNC_CUDA_TRY(cudaGraphLaunch(g.exec[2], g.cs));
      kernels += kn[2];
      t += kSweepsPerGraph;
    } else if (sampled) {
      const int j = t / kProfileEvery;
      if (j == 0) {
        NNC_TRY(prof.init(samples));
        NNC_TRY(capture_sweep<T>(X, F, G, b, eps, trace, prof.capture_events(), tcp, true, g, 1));
        NNC_TRY(prof.bind(g.graph[1]));
        NNC_TRY(count_kernel_nodes(g.graph[1], &kn[1]));
      }
      NNC_TRY(prof.set_launch(g.exec[1], j));
      NNC_CUDA_TRY(cudaGraphLaunch(g.exec[1], g.cs));
      kernels += kn[1];
      ++t;
    } else {
      NNC_CUDA_TRY(cudaGraphLaunch(g.exec[0], g.cs));
      kernels += kn[0];
      ++t;
    }
    if (checkpoints && ck->at(first + t - 1)) {
      const int sweep = first + t - 1;
      NNC_TRY(launch_sweep_core<T>(F, G, b, eps, trace, 1, tcp, g.cs));
      const T* fac[3] = {F[0], F[1], F[2]};
      NNC_TRY(residual_run<T>(ck->X, 3, ck->dims, 0, ck->m, 0, fac, G, *ck->rw, nullptr,
                              trace + sweep, g.cs));
      if (ck->tol > 0.0) {
        double e = 0.0;
        NNC_CUDA_TRY(cudaMemcpyAsync(&e, trace + sweep, sizeof(double), cudaMemcpyDeviceToHost,
                                     g.cs));
        NNC_CUDA_TRY(cudaStreamSynchronize(g.cs));
        bool stop = false;
        if (ck->last > 0.0 && e > 0.0) {
          const double drop = (ck->last - e) / e;
          ck->peak = drop > ck->peak ? drop : ck->peak;
          stop = drop < ck->tol * ck->peak;
        }
        ck->last = e;
        if (stop) break;
      }
    }
  }
  *done = t;
  note_graph_launches(kernels);
  NNC_TRY(launch_sweep_core<T>(F, G, b, eps, trace ? trace : b.trace_dummy, trace ? 1 : 0, tcp,
                               g.cs));
  NNC_CUDA_TRY(cudaEventRecord(g.join, g.cs));
  NNC_CUDA_TRY(cudaStreamWaitEvent(s, g.join, 0));
  NNC_CUDA_TRY(cudaStreamSynchronize(g.cs));
  if (samples > 0) NNC_TRY(prof.collect(t / kProfileEvery < samples ? t / kProfileEvery : samples));
  return NNC_OK;
}

// passes: 0 = SIMT for every sweep; 1 = TF32x3 tensor cores for every sweep
// (FP32-accurate); 2 = BF16 tensor cores, then TF32x3 for the refinement sweeps.
// A tensor-core plan that the shape does not allow falls back to SIMT passes.
template <typename T>
int ntd_fit3_impl(const T* X, const int64_t* dims, const int* m, const nnc_opts* o, T* const* F,
                  T* G, double* trace, double* rel_err, int passes, int* refined_from,
                  cudaStream_t s) {
  const int64_t N1 = dims[0], N2 = dims[1], N3 = dims[2];
  const int m1 = m[0], m2 = m[1], m3 = m[2];
  const int64_t nX = N1 * N2 * N3;
  const int64_t nc = (int64_t)m1 * m2 * m3;
  Scratch sc(s);
  NtdState<T> b{};
  for (int k = 0; k < 3; ++k) {
    b.N[k] = dims[k];
    b.m[k] = m[k];
  }

  NNC_TRY(sc.get(&b.stats_part, 3 * kStatBlocks));
  NNC_TRY(sc.get(&b.stats, 3));
  NNC_TRY(sc.get(&b.trace_dummy, 1));
  NNC_TRY(sc.get(&b.resid2, 2));
  NNC_TRY(sc.get(&b.counter, 2));
  NNC_TRY(sc.get(&b.dots, 2 * (size_t)m[0]));
  NNC_TRY(sc.get(&b.done, 1));
  NNC_TRY(sc.get(&b.gate, 1));
  NNC_CUDA_TRY(launch_tensor_stats<T>(X, nX, b.stats_part, b.stats, s));
  double st[3];
  NNC_CUDA_TRY(cudaMemcpyAsync(st, b.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (st[2] > 0.0) return NNC_ERR_NONFINITE;
  if (st[1] > 0.0) return NNC_ERR_NEGATIVE_INPUT;
  if (!(st[0] > 0.0)) return NNC_ERR_INVALID_ARG;  // X == 0: the relative error is undefined


  NNC_TRY(sc.get(&b.P3, (size_t)(N1 * N2 * m3)));
  NNC_TRY(sc.get(&b.P1, (size_t)(m1 * N2 * N3)));
  NNC_TRY(sc.get(&b.Y3, (size_t)((int64_t)m1 * m2 * N3)));
  NNC_TRY(sc.get(&b.num2, (size_t)(N2 * m2)));
  NNC_TRY(sc.get(&b.num3, (size_t)(N3 * m3)));
  NNC_TRY(sc.get(&b.Yb, (size_t)std::max(N1 * m2 * m3, N2 * m1 * m3)));
  NNC_TRY(sc.get(&b.M, (size_t)nc));
  NNC_TRY(sc.get(&b.W1, (size_t)nc));
  NNC_TRY(sc.get(&b.W3, (size_t)nc));
  NNC_TRY(sc.get(&b.G2, (size_t)nc));
  NNC_TRY(sc.get(&b.G3, (size_t)nc));
  for (int k = 0; k < 3; ++k) {
    NNC_TRY(sc.get(&b.S[k], (size_t)(m[k] * m[k])));
    NNC_TRY(sc.get(&b.H[k], (size_t)(m[k] * m[k])));
  }

  tc::TcPlan plan16, plan32;
  const tc::TcPlan* fast = nullptr;   // the first iters - refine sweeps
  const tc::TcPlan* exact = nullptr;  // FP32-accurate sweeps
  // The refinement trigger may end the fast sweeps early (exact checkpoints needed).
  const bool trigger = passes == 2 && o->refine_tol > 0.0 && o->exact_every > 0 && trace;
  if constexpr (std::is_same<T, float>::value) {
    if (passes == 2 && o->iters > o->refine_iters) {
      NNC_TRY(plan16.init(tc::kKindBf16, X, N1, N2, N3, m1, m3, sc, s, /*p1_kj=*/true));
      // The BF16 passes stream X about twice as fast as the TF32x3 ones and
      // the small kernels beside them would otherwise hold SMs the pass
      // waits for: they leave 32 SMs to them (measured at 512^3, m = 32: 258
      // -> 225 us per sweep; the TF32x3 sweep is fastest with every SM).
      plan16.reserve_sms = 32;
      fast = &plan16;
    }
    if (passes >= 1 && (passes == 1 || o->refine_iters > 0 || trigger)) {
      const int st = plan32.init(tc::kKindTf32x3, X, N1, N2, N3, m1, m3, sc, s, /*p1_kj=*/true);
      if (st == NNC_OK) exact = &plan32;
      else if (st != NNC_ERR_UNSUPPORTED) return st;
    }
  }
  const int n_fast_max = fast ? o->iters - o->refine_iters : 0;
  if (!exact && (o->iters - n_fast_max > 0 || trigger))
    NNC_TRY(sc.get(&b.P1s, (size_t)(m1 * N2 * N3)));
  ResidualWork<T> rw;
  Checkpoints<T> ck;
  if (o->exact_every > 0 && trace) {
    NNC_TRY(residual_prepare<T>(3, dims, 0, m, 0, sc, &rw));
    ck.every = o->exact_every;
    ck.total = o->iters;
    ck.X = X;
    ck.dims = dims;
    ck.m = m;
    ck.rw = &rw;
  }
  if constexpr (std::is_same<T, float>::value) {
    // The tensor-core passes form the shares of Y1 when the shape allows it
    // (y1_fusable), the TF32x3 passes also those of Y3 (y3_fusable).
    const tc::TcPlan* any = exact ? exact : fast;
    if (any && any->y1_fusable(m2)) {
      b.y_nh = (int)(N2 / 128);
      NNC_TRY(sc.get(&b.Y1p, (size_t)(N1 * b.y_nh) * m2 * m3));
    }
    if ((exact && exact->y3_fusable(m2)) || (fast && fast->y3_fusable(m2))) {
      b.y_nh = (int)(N2 / 128);
      NNC_TRY(sc.get(&b.Y3p, (size_t)(N3 * b.y_nh) * m1 * m2));
    }
  }

  // Prologue: S_k = F_k^T F_k, H1 = unfold_1(G x_2 S2 x_3 S3) unfold_1(G)^T,
  // the BF16 operand of F^(3), the trace counter.
  for (int k = 0; k < 3; ++k) NNC_TRY(launch_gram<T>(F[k], dims[k], m[k], b.S[k], s));
  NNC_TRY(launch_permute_core<T>(G, m1, m2, m3, b.G2, b.G3, s));
  {
    HArgs<T> h{};
    h.Gn = G;  h.mp = m1;  h.mu = m2;  h.mv = m3;
    h.su = b.S[1];  h.sv = b.S[2];  h.H = b.H[0];
    NNC_TRY(launch_hmat<T>(h, s));
  }
  if constexpr (std::is_same<T, float>::value) {
    if (fast) NNC_TRY(fast->convert_b3(F[2], s));
    if (exact && !fast) NNC_TRY(exact->convert_b3(F[2], s));
  }
  NNC_CUDA_TRY(cudaMemsetAsync(b.counter, 0, 2 * sizeof(int), s));
  NNC_CUDA_TRY(cudaMemsetAsync(b.done, 0, sizeof(int), s));
  NNC_CUDA_TRY(cudaMemsetAsync(b.gate, 0, sizeof(int), s));

  int n_fast = 0;
  ck.tol = trigger ? o->refine_tol : 0.0;
  NNC_TRY(run_sweeps<T>(X, F, G, b, o->eps, trace, n_fast_max, 0, &ck, fast, s, &n_fast));
  if (fast) NNC_TRY(fast->check(s));
  if (refined_from) *refined_from = n_fast;
  ck.tol = 0.0;
  if constexpr (std::is_same<T, float>::value) {
    // The FP32-accurate sweeps start from the factors the fast sweeps left.
    if (exact && fast && o->iters - n_fast > 0) NNC_TRY(exact->convert_b3(F[2], s));
  }
  int n_rest = 0;
  NNC_TRY(run_sweeps<T>(X, F, G, b, o->eps, trace, o->iters - n_fast, n_fast, &ck, exact, s,
                        &n_rest));
  if (exact) NNC_TRY(exact->check(s));
  NNC_TRY(check_trace_finite(b.counter, s, "ntd_fit"));

  if (rel_err) {
    const T* fac[3] = {F[0], F[1], F[2]};
    NNC_TRY(residual_device<T>(X, 3, dims, 0, m, 0, fac, G, b.resid2, sc, s));
    double h[2];
    NNC_CUDA_TRY(cudaMemcpyAsync(h, b.resid2, sizeof(h), cudaMemcpyDeviceToHost, s));
    NNC_CUDA_TRY(cudaStreamSynchronize(s));
    *rel_err = sqrt(h[0] / h[1]);
  }
  return NNC_OK;
}

}  // namespace

template <typename T>
int ntd_fit3(const T* X, const int64_t* dims, const int* m, const nnc_opts* o, T* const* F, T* G,
             double* trace, double* rel_err, bool tensor_cores, cudaStream_t s) {
  return ntd_fit3_impl<T>(X, dims, m, o, F, G, trace, rel_err, tensor_cores ? 1 : 0, nullptr, s);
}

int ntd_fit3_bf16(const float* X, const int64_t* dims, const int* m, const nnc_opts* o,
                  float* const* F, float* G, double* trace, double* rel_err, int* refined_from,
                  cudaStream_t s) {
  return ntd_fit3_impl<float>(X, dims, m, o, F, G, trace, rel_err, 2, refined_from, s);
}

template int ntd_fit3<float>(const float*, const int64_t*, const int*, const nnc_opts*,
                             float* const*, float*, double*, double*, bool, cudaStream_t);
template int ntd_fit3<double>(const double*, const int64_t*, const int*, const nnc_opts*,
                              double* const*, double*, double*, double*, bool, cudaStream_t);

}  // namespace nnc
