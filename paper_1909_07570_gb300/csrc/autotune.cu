// Launch-shape autotuner of the one-block-per-job batched kernels.
//
// A batched fit runs one thread block per job. The best block size depends on
// the jobs: tiny cores leave most of 256 threads idle and fit four times as
// many blocks per SM at 64 threads; larger ones want the threads. The
// candidates are tried on the fit itself (see run_tuned), so tuning costs one
// host wait per new shape class and no extra sweeps.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "autotune.cuh"

namespace nnc {
namespace {

constexpr int kCandidates[] = {32, 64, 128, 256};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

std::atomic<bool> g_on{true};
std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_cache;  // (device, key) -> threads

std::tuple<int, int, int, int, int> full_key(const TuneKey& k) {
  int dev = 0;
  cudaGetDevice(&dev);
  return std::make_tuple(dev, k.kernel, k.elem, k.work, k.jobs);
}

bool lookup(const TuneKey& key, int* threads) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(full_key(key));
  if (it == g_cache.end()) return false;
  *threads = it->second;
  return true;
}

struct Events {
  std::vector<cudaEvent_t> ev;
  ~Events() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

}  // namespace

int size_class(long long n) {
  int c = 0;
  while (n > 1) {
    n = (n + 1) >> 1;
    ++c;
  }
  return c;
}

void autotune_set(bool on) { g_on.store(on); }
bool autotune_on() { return g_on.load(); }

int tuned_threads(const TuneKey& key, int default_threads) {
  int t = default_threads;
  if (g_on.load()) lookup(key, &t);
  return t;
}

int run_tuned(const TuneKey& key, int iters, int default_threads, cudaStream_t s,
              const TunedLaunch& launch) {
  int threads = default_threads;
  if (!g_on.load() || lookup(key, &threads)) return launch(threads, iters, true);
  // Trial sweeps per candidate, plus one warm-up launch at the default size
  // (the first launch of a batch pays for cold caches); at least one sweep is
  // left for the final launch.
  int per = iters / 32;
  per = per > 16 ? 16 : per;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  NNC_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (per < 2 || (kNumCandidates + 1) * per >= iters || cap != cudaStreamCaptureStatusNone)
    return launch(threads, iters, true);
  Events e;
  e.ev.assign(2 * kNumCandidates, nullptr);
  for (cudaEvent_t& ev : e.ev) NNC_CUDA_TRY(cudaEventCreate(&ev));
  NNC_TRY(launch(default_threads, per, false));
  for (int c = 0; c < kNumCandidates; ++c) {
    NNC_CUDA_TRY(cudaEventRecord(e.ev[2 * c], s));
    NNC_TRY(launch(kCandidates[c], per, false));
    NNC_CUDA_TRY(cudaEventRecord(e.ev[2 * c + 1], s));
  }
  NNC_CUDA_TRY(cudaEventSynchronize(e.ev[2 * kNumCandidates - 1]));
  float best = 0.0f;
  for (int c = 0; c < kNumCandidates; ++c) {
    float ms = 0.0f;
    NNC_CUDA_TRY(cudaEventElapsedTime(&ms, e.ev[2 * c], e.ev[2 * c + 1]));
    if (c == 0 || ms < best) {
      best = ms;
      threads = kCandidates[c];
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[full_key(key)] = threads;
  }
  return launch(threads, iters - (kNumCandidates + 1) * per, true);
}

}  // namespace nnc
