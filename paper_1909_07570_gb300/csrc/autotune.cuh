// Launch-shape autotuner of the one-block-per-job batched kernels (autotune.cu).
#pragma once

#include <functional>

#include "common.cuh"

namespace nnc {

// The kernel family and the shape classes a choice is cached under.
enum TuneKernel { kTuneNncp = 0, kTuneNtdSmall, kTuneNtdL2, kTuneCpxL2, kTuneNmfSmall };

struct TuneKey {
  int kernel;    // TuneKernel
  int elem;      // sizeof(T)
  int work;      // log2 class of the largest job's per-sweep work (or state size)
  int jobs;      // log2 class of the number of jobs
};

// launch(threads, sweeps, last): queues one launch of `sweeps` sweeps of every
// job on the stream with `threads` threads per block; `last` marks the launch
// that must write the jobs' final outputs (relative errors).
using TunedLaunch = std::function<int(int threads, int sweeps, bool last)>;

// Runs `iters` sweeps through `launch`. The kernels this serves give results
// that depend neither on the block size nor on how the sweeps are split over
// launches (each launch reloads the state the previous one stored, and every
// sum has a fixed order). So, on the first call for a key with enough sweeps
// (and a stream that is not being captured), the first sweeps go to trial
// launches, one per candidate block size, timed with events (one host wait);
// the fit proceeds through them. The rest runs at the fastest candidate, which
// is cached for the key. Otherwise one launch at the cached (or default) size.
int run_tuned(const TuneKey& key, int iters, int default_threads, cudaStream_t s,
              const TunedLaunch& launch);

// The cached block size for `key`, or `default_threads`; never times anything.
int tuned_threads(const TuneKey& key, int default_threads);

// log2 class of a positive count (0 for n <= 1).
int size_class(long long n);

void autotune_set(bool on);
bool autotune_on();

}  // namespace nnc
