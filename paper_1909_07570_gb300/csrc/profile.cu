// Event timing of the passes over X (see profile.cuh) and its C ABI.
#include <map>
#include <mutex>

#include "profile.cuh"

namespace nnc {
namespace {

std::mutex g_mu;
bool g_on = false;
long long g_launches[kProfileKinds] = {};
double g_ms[kProfileKinds] = {};
// Per-device event pool. Events [0, cursor) are handed out since the last
// read; their (start, stop, kind) triples wait in g_pending until
// nnc_profile_read resolves them, so no elapsed time is read inside a call.
struct Pool {
  std::vector<cudaEvent_t> ev;
  size_t cursor = 0;
};
std::map<int, Pool> g_pool;
struct Pending {
  int dev;
  cudaEvent_t start, stop;
  int kind;
};
std::vector<Pending> g_pending;

int resolve_pending_locked() {
  if (g_pending.empty()) return NNC_OK;
  int cur = 0;
  NNC_CUDA_TRY(cudaGetDevice(&cur));
  for (const Pending& p : g_pending) {
    NNC_CUDA_TRY(cudaSetDevice(p.dev));
    NNC_CUDA_TRY(cudaEventSynchronize(p.stop));
    float v = 0.f;
    NNC_CUDA_TRY(cudaEventElapsedTime(&v, p.start, p.stop));
    g_launches[p.kind] += 1;
    g_ms[p.kind] += v;
  }
  NNC_CUDA_TRY(cudaSetDevice(cur));
  g_pending.clear();
  for (auto& kv : g_pool) kv.second.cursor = 0;
  return NNC_OK;
}

}  // namespace

bool profile_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

int PassProfiler::init(int launches) {
  int dev = 0;
  NNC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Pool& pool = g_pool[dev];
  const size_t need = 4 * (size_t)(launches > 0 ? launches : 1);
  while (pool.ev.size() < pool.cursor + need) {
    cudaEvent_t e;
    NNC_CUDA_TRY(cudaEventCreate(&e));
    pool.ev.push_back(e);
  }
  ev_.assign(pool.ev.begin() + pool.cursor, pool.ev.begin() + pool.cursor + need);
  pool.cursor += need;
  dev_ = dev;
  cap_.start[0] = ev_[0];
  cap_.stop[0] = ev_[1];
  cap_.start[1] = ev_[2];
  cap_.stop[1] = ev_[3];
  return NNC_OK;
}

int PassProfiler::bind(cudaGraph_t graph) {
  size_t n = 0;
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  NNC_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &n));
  int found = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    NNC_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t e;
    NNC_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &e));
    for (int k = 0; k < 4; ++k)
      if (e == ev_[k]) {
        node_[k] = nd;
        ++found;
      }
  }
  if (found != 4) {
    set_error_detail_text("profiler: event-record nodes not found in the captured sweep");
    return NNC_ERR_CUDA;
  }
  return NNC_OK;
}

int PassProfiler::set_launch(cudaGraphExec_t exec, int t) {
  if (t == 0) return NNC_OK;  // the captured nodes already hold launch 0's events
  for (int k = 0; k < 4; ++k)
    NNC_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(exec, node_[k], ev_[4 * (size_t)t + k]));
  return NNC_OK;
}

int PassProfiler::collect(int launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int t = 0; t < launches; ++t)
    for (int p = 0; p < 2; ++p)
      g_pending.push_back({dev_, ev_[4 * (size_t)t + 2 * p], ev_[4 * (size_t)t + 2 * p + 1],
                           kind_base_ + p});
  return NNC_OK;
}

}  // namespace nnc

extern "C" {

int nnc_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(nnc::g_mu);
  nnc::g_on = on != 0;
  nnc::g_pending.clear();
  for (auto& kv : nnc::g_pool) kv.second.cursor = 0;
  for (int k = 0; k < nnc::kProfileKinds; ++k) {
    nnc::g_launches[k] = 0;
    nnc::g_ms[k] = 0.0;
  }
  return NNC_OK;
}

int nnc_profile_read(int kind, long long* launches, double* total_ms) {
  if (kind < 0 || kind >= nnc::kProfileKinds || launches == nullptr || total_ms == nullptr)
    return NNC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(nnc::g_mu);
  NNC_TRY(nnc::resolve_pending_locked());
  *launches = nnc::g_launches[kind];
  *total_ms = nnc::g_ms[kind];
  return NNC_OK;
}

}  // extern "C"
