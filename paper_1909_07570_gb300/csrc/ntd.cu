// nnTD of a 3-way tensor (Alg. 1, step 1) on the GPU: the sweep loop.
//
// One sweep (Gauss-Seidel: F^(1), F^(2), F^(3), then G), with S_k = F^(k)T F^(k)
// and the unfolding identity Eq. unfolding:property:
//   P3 = X x_3 F^(3)T                       first pass over X
//   Y1 = P3 x_2 F^(2)T        Num_1 = unfold_1(Y1) unfold_1(G)^T
//   H1 = unfold_1(G x_2 S2 x_3 S3) unfold_1(G)^T,  Den_1 = F^(1) H1;  MU on F^(1)
//   Y2 = P3 x_1 F^(1)T (new F^(1))          Num_2, H2 likewise;   MU on F^(2)
//   P1 = X x_1 F^(1)T                       second pass over X (new F^(1))
//   Y3 = P1 x_2 F^(2)T (new F^(2))          Num_3, H3;            MU on F^(3)
//   M  = Y3 x_3 F^(3)T = X x_1 F^(1)T x_2 F^(2)T x_3 F^(3)T
//   G <- max(G * M / max(G x_1 S1 x_2 S2 x_3 S3, eps), 0)
//   trace = sqrt(||X||^2 - 2<M, G> + <G, G x_k S_k>) / ||X||   (FP64 sums)
// X is read twice per sweep; every other array is at most N^2 m.
//
// Core-sized products are shared where the factors they use have not changed:
// W3 = G x_1 S1 x_2 S2 serves H3 and, times S3, the core denominator; and
// W1 = G_new x_2 S2 x_3 S3 serves the residual (times S1) and the next
// sweep's H1.
//
// The sweep is captured once as a CUDA graph on a private stream and replayed
// `iters` times; the trace slot advances through a device counter.
//
// NNC_BF16_REFINE: the two passes over X run on the tensor cores from a BF16
// copy of X (tc_ttm.cu) for the first iters - refine_iters sweeps; the last
// refine_iters sweeps replay the FP32 graph on X itself. Everything but the two
// passes is FP32 in both.
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "ntd.cuh"
#include "profile.cuh"
#include "residual.cuh"
#include "tc_ttm.cuh"

namespace nnc {

namespace {

template <typename T>
struct NtdBuffers {
  T *P3, *P1, *Y1, *Y2, *Y3, *M, *W1, *W, *Wt, *D, *S[3], *H, *Num, *split;
  size_t split_cap;
  double *stats_part, *stats, *trace_dummy, *resid2;
  int* counter;
};

template <typename T>
int pass_x3(const T* X, int64_t N1, int64_t N2, int64_t N3, int m3, const T* F3, T* P3,
            NtdBuffers<T>& b, const tc::TcPlan* tcp, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (tcp) return tcp->pass3(F3, P3, s);
  }
  NNC_CUDA_TRY(launch_ttm<T>(X, N1 * N2, (int)N3, 1, F3, m3, 1, m3, P3, b.split, b.split_cap, s));
  return NNC_OK;
}

template <typename T>
int pass_x1(const T* X, int64_t N1, int64_t N2, int64_t N3, int m1, const T* F1, T* P1,
            NtdBuffers<T>& b, const tc::TcPlan* tcp, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (tcp) return tcp->pass1(F1, P1, s);
  }
  NNC_CUDA_TRY(launch_ttm<T>(X, 1, (int)N1, N2 * N3, F1, m1, 1, m1, P1, b.split, b.split_cap, s));
  return NNC_OK;
}

template <typename T>
int sweep3(const T* X, const int64_t* N, const int* m, T* const* F, T* G, NtdBuffers<T>& b,
           double eps, double* trace, int trace_stride, const PassEvents* ev,
           const tc::TcPlan* tcp, cudaStream_t s) {
  const int64_t N1 = N[0], N2 = N[1], N3 = N[2];
  const int m1 = m[0], m2 = m[1], m3 = m[2];
  const int64_t nc = (int64_t)m1 * m2 * m3;
  T* sp = b.split;
  const size_t cap = b.split_cap;

  // ---- mode 1 ------------------------------------------------------------
  // P3[i, j, c] = sum_k X[i, j, k] F3[k, c]
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->start[0], s, cudaEventRecordExternal));
  NNC_TRY(pass_x3<T>(X, N1, N2, N3, m3, F[2], b.P3, b, tcp, s));
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->stop[0], s, cudaEventRecordExternal));
  // Y1[i, b, c] = sum_j F2[j, b] P3[i, j, c]
  NNC_CUDA_TRY(launch_ttm<T>(b.P3, N1, (int)N2, m3, F[1], m2, 1, m2, b.Y1, sp, cap, s));
  // H1 = unfold_1(W1) unfold_1(G)^T with W1 = G x_2 S2 x_3 S3 (kept from the last sweep)
  NNC_CUDA_TRY(launch_pair_contract<T>(b.W1, G, 1, m1, m1, (int64_t)m2 * m3, b.H, s));
  // Num_1[i, a] = sum_{b,c} Y1[i, b, c] G[a, b, c]
  NNC_CUDA_TRY(launch_pair_contract<T>(b.Y1, G, 1, (int)N1, m1, (int64_t)m2 * m3, b.Num, s));
  NNC_CUDA_TRY(launch_factor_mu<T>(F[0], b.Num, b.H, N1, m1, eps, s));
  NNC_CUDA_TRY(launch_ttm<T>(F[0], 1, (int)N1, m1, F[0], m1, 1, m1, b.S[0], sp, cap, s));

  // ---- mode 2 ------------------------------------------------------------
  // Y2[a, j, c] = sum_i F1[i, a] P3[i, j, c]
  NNC_CUDA_TRY(launch_ttm<T>(b.P3, 1, (int)N1, N2 * m3, F[0], m1, 1, m1, b.Y2, sp, cap, s));
  // W = G x_1 S1 x_3 S3;  H2 = unfold_2(W) unfold_2(G)^T
  NNC_CUDA_TRY(launch_ttm<T>(G, 1, m1, (int64_t)m2 * m3, b.S[0], m1, 1, m1, b.Wt, sp, cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(b.Wt, (int64_t)m1 * m2, m3, 1, b.S[2], m3, 1, m3, b.W, sp, cap, s));
  NNC_CUDA_TRY(launch_pair_contract<T>(b.W, G, m1, m2, m2, m3, b.H, s));
  // Num_2[j, b] = sum_{a,c} Y2[a, j, c] G[a, b, c]
  NNC_CUDA_TRY(launch_pair_contract<T>(b.Y2, G, m1, (int)N2, m2, m3, b.Num, s));
  NNC_CUDA_TRY(launch_factor_mu<T>(F[1], b.Num, b.H, N2, m2, eps, s));
  NNC_CUDA_TRY(launch_ttm<T>(F[1], 1, (int)N2, m2, F[1], m2, 1, m2, b.S[1], sp, cap, s));

  // ---- mode 3 ------------------------------------------------------------
  // P1[a, j, k] = sum_i F1[i, a] X[i, j, k]
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->start[1], s, cudaEventRecordExternal));
  NNC_TRY(pass_x1<T>(X, N1, N2, N3, m1, F[0], b.P1, b, tcp, s));
  if (ev) NNC_CUDA_TRY(cudaEventRecordWithFlags(ev->stop[1], s, cudaEventRecordExternal));
  // Y3[a, b, k] = sum_j F2[j, b] P1[a, j, k]
  NNC_CUDA_TRY(launch_ttm<T>(b.P1, m1, (int)N2, N3, F[1], m2, 1, m2, b.Y3, sp, cap, s));
  // W3 = G x_1 S1 x_2 S2 (into W);  H3 = unfold_3(W3) unfold_3(G)^T
  NNC_CUDA_TRY(launch_ttm<T>(G, 1, m1, (int64_t)m2 * m3, b.S[0], m1, 1, m1, b.Wt, sp, cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(b.Wt, m1, m2, m3, b.S[1], m2, 1, m2, b.W, sp, cap, s));
  NNC_CUDA_TRY(launch_pair_contract<T>(b.W, G, (int64_t)m1 * m2, m3, m3, 1, b.H, s));
  // Num_3[k, c] = sum_{a,b} Y3[a, b, k] G[a, b, c]
  NNC_CUDA_TRY(launch_pair_contract<T>(b.Y3, G, (int64_t)m1 * m2, (int)N3, m3, 1, b.Num, s));
  NNC_CUDA_TRY(launch_factor_mu<T>(F[2], b.Num, b.H, N3, m3, eps, s));
  NNC_CUDA_TRY(launch_ttm<T>(F[2], 1, (int)N3, m3, F[2], m3, 1, m3, b.S[2], sp, cap, s));

  // ---- core --------------------------------------------------------------
  // M[a, b, c] = sum_k Y3[a, b, k] F3[k, c]
  NNC_CUDA_TRY(launch_ttm<T>(b.Y3, (int64_t)m1 * m2, (int)N3, 1, F[2], m3, 1, m3, b.M, sp, cap, s));
  // D = W3 x_3 S3 = G x_1 S1 x_2 S2 x_3 S3
  NNC_CUDA_TRY(launch_ttm<T>(b.W, (int64_t)m1 * m2, m3, 1, b.S[2], m3, 1, m3, b.D, sp, cap, s));
  NNC_CUDA_TRY(launch_elementwise_mu<T>(G, b.M, b.D, nc, eps, s));
  // W1 = G x_2 S2 x_3 S3 with the new G (next sweep's H1); D = W1 x_1 S1
  NNC_CUDA_TRY(launch_ttm<T>(G, m1, m2, m3, b.S[1], m2, 1, m2, b.Wt, sp, cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(b.Wt, (int64_t)m1 * m2, m3, 1, b.S[2], m3, 1, m3, b.W1, sp, cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(b.W1, 1, m1, (int64_t)m2 * m3, b.S[0], m1, 1, m1, b.D, sp, cap, s));
  NNC_CUDA_TRY(launch_residual_identity<T>(b.M, G, b.D, nc, b.stats, trace, trace_stride,
                                           b.counter, s));
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

// RAII holder of the private stream, graph and events of one ntd_fit call.
struct GraphRun {
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ~GraphRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (cs) cudaStreamDestroy(cs);
  }
};

// Captures one sweep on a private stream and replays it `count` times after
// the work already queued on `s`; `s` then waits for the replays.
template <typename T>
int run_sweeps(const T* X, const int64_t* dims, const int* m, T* const* F, T* G,
               NtdBuffers<T>& b, double eps, double* trace, int count, const tc::TcPlan* tcp,
               cudaStream_t s) {
  if (count <= 0) return NNC_OK;
  GraphRun g;
  NNC_CUDA_TRY(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
  NNC_CUDA_TRY(cudaEventRecord(g.fork, s));
  NNC_CUDA_TRY(cudaStreamWaitEvent(g.cs, g.fork, 0));

  PassProfiler prof(tcp ? 2 : 0);
  const PassEvents* capture_ev = nullptr;
  if (profile_enabled()) {
    NNC_TRY(prof.init(count));
    capture_ev = prof.capture_events();
  }
  NNC_CUDA_TRY(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
  const int cap_st = sweep3<T>(X, dims, m, F, G, b, eps, trace ? trace : b.trace_dummy,
                               trace ? 1 : 0, capture_ev, tcp, g.cs);
  const cudaError_t end_e = cudaStreamEndCapture(g.cs, &g.graph);
  if (cap_st != NNC_OK) return cap_st;
  NNC_CUDA_TRY(end_e);
  NNC_CUDA_TRY(cudaGraphInstantiate(&g.exec, g.graph, 0));
  long long kernel_nodes = 0;
  NNC_TRY(count_kernel_nodes(g.graph, &kernel_nodes));
  if (capture_ev) NNC_TRY(prof.bind(g.graph));
  for (int t = 0; t < count; ++t) {
    if (capture_ev) NNC_TRY(prof.set_launch(g.exec, t));
    NNC_CUDA_TRY(cudaGraphLaunch(g.exec, g.cs));
  }
  note_graph_launches(kernel_nodes * count);
  NNC_CUDA_TRY(cudaEventRecord(g.join, g.cs));
  NNC_CUDA_TRY(cudaStreamWaitEvent(s, g.join, 0));
  NNC_CUDA_TRY(cudaStreamSynchronize(g.cs));
  if (capture_ev) NNC_TRY(prof.collect(count));
  return NNC_OK;
}

template <typename T>
int ntd_fit3_impl(const T* X, const int64_t* dims, const int* m, const nnc_opts* o, T* const* F,
                  T* G, double* trace, double* rel_err, bool use_tc, cudaStream_t s) {
  const int64_t N1 = dims[0], N2 = dims[1], N3 = dims[2];
  const int m1 = m[0], m2 = m[1], m3 = m[2];
  const int64_t nX = N1 * N2 * N3;
  Scratch sc(s);
  NtdBuffers<T> b{};
  const int64_t nc = (int64_t)m1 * m2 * m3;
  const int64_t mmax = m1 > m2 ? (m1 > m3 ? m1 : m3) : (m2 > m3 ? m2 : m3);
  const int64_t Nmax = N1 > N2 ? (N1 > N3 ? N1 : N3) : (N2 > N3 ? N2 : N3);
  const int64_t nY1 = N1 * m2 * m3, nY2 = (int64_t)m1 * N2 * m3, nY3 = (int64_t)m1 * m2 * N3;
  int64_t ymax = nY1 > nY2 ? nY1 : nY2;
  ymax = ymax > nY3 ? ymax : nY3;
  ymax = ymax > nc ? ymax : nc;
  b.split_cap = (size_t)(8 * ymax > (1 << 20) ? 8 * ymax : (1 << 20));

  NNC_TRY(sc.get(&b.stats_part, 3 * kStatBlocks));
  NNC_TRY(sc.get(&b.stats, 3));
  NNC_TRY(sc.get(&b.trace_dummy, 1));
  NNC_TRY(sc.get(&b.resid2, 2));
  NNC_TRY(sc.get(&b.counter, 1));
  NNC_CUDA_TRY(launch_tensor_stats<T>(X, nX, b.stats_part, b.stats, s));
  double st[3];
  NNC_CUDA_TRY(cudaMemcpyAsync(st, b.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (st[2] > 0.0) return NNC_ERR_NONFINITE;
  if (st[1] > 0.0) return NNC_ERR_NEGATIVE_INPUT;
  if (!(st[0] > 0.0)) return NNC_ERR_INVALID_ARG;  // X == 0: the relative error is undefined

  NNC_TRY(sc.get(&b.P3, (size_t)(N1 * N2 * m3)));
  NNC_TRY(sc.get(&b.P1, (size_t)(m1 * N2 * N3)));
  NNC_TRY(sc.get(&b.Y1, (size_t)nY1));
  NNC_TRY(sc.get(&b.Y2, (size_t)nY2));
  NNC_TRY(sc.get(&b.Y3, (size_t)nY3));
  NNC_TRY(sc.get(&b.M, (size_t)nc));
  NNC_TRY(sc.get(&b.W1, (size_t)nc));
  NNC_TRY(sc.get(&b.W, (size_t)nc));
  NNC_TRY(sc.get(&b.Wt, (size_t)nc));
  NNC_TRY(sc.get(&b.D, (size_t)nc));
  for (int k = 0; k < 3; ++k) NNC_TRY(sc.get(&b.S[k], (size_t)(m[k] * m[k])));
  NNC_TRY(sc.get(&b.H, (size_t)(mmax * mmax)));
  NNC_TRY(sc.get(&b.Num, (size_t)(Nmax * mmax)));
  NNC_TRY(sc.get(&b.split, b.split_cap));

  tc::TcPlan plan;
  const tc::TcPlan* tcp = nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (use_tc && o->iters > o->refine_iters) {
      NNC_TRY(plan.init(X, N1, N2, N3, m1, m3, sc, s));
      tcp = &plan;
    }
  }

  // Prologue: Grams, W1 = G x_2 S2 x_3 S3, trace counter.
  for (int k = 0; k < 3; ++k)
    NNC_CUDA_TRY(launch_ttm<T>(F[k], 1, (int)dims[k], m[k], F[k], m[k], 1, m[k], b.S[k], b.split,
                               b.split_cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(G, m1, m2, m3, b.S[1], m2, 1, m2, b.Wt, b.split, b.split_cap, s));
  NNC_CUDA_TRY(launch_ttm<T>(b.Wt, (int64_t)m1 * m2, m3, 1, b.S[2], m3, 1, m3, b.W1, b.split,
                             b.split_cap, s));
  NNC_CUDA_TRY(cudaMemsetAsync(b.counter, 0, sizeof(int), s));

  const int n_fast = tcp ? o->iters - o->refine_iters : 0;
  NNC_TRY(run_sweeps<T>(X, dims, m, F, G, b, o->eps, trace, n_fast, tcp, s));
  if (tcp) NNC_TRY(plan.check(s));
  NNC_TRY(run_sweeps<T>(X, dims, m, F, G, b, o->eps, trace, o->iters - n_fast, nullptr, s));

  if (rel_err) {
    const T* fac[3] = {F[0], F[1], F[2]};
    NNC_TRY(residual3_device<T>(X, dims, 0, m, 0, fac, G, b.resid2, sc, s));
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
             double* trace, double* rel_err, cudaStream_t s) {
  return ntd_fit3_impl<T>(X, dims, m, o, F, G, trace, rel_err, false, s);
}

int ntd_fit3_bf16(const float* X, const int64_t* dims, const int* m, const nnc_opts* o,
                  float* const* F, float* G, double* trace, double* rel_err, cudaStream_t s) {
  return ntd_fit3_impl<float>(X, dims, m, o, F, G, trace, rel_err, true, s);
}

template int ntd_fit3<float>(const float*, const int64_t*, const int*, const nnc_opts*,
                             float* const*, float*, double*, double*, cudaStream_t);
template int ntd_fit3<double>(const double*, const int64_t*, const int*, const nnc_opts*,
                              double* const*, double*, double*, double*, cudaStream_t);

}  // namespace nnc
