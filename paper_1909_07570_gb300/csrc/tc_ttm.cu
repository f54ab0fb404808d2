// Tensor-core (tcgen05) mode products: the two passes over X of an nnTD sweep
// (n-mode multiplication, Appendix A), in two number formats.
//
//   BF16    X is kept as a BF16 copy Xb with per-slice power-of-two scales s_i
//           (mode-1 slices), rows padded with zeros to Kp = roundup(N3, 64):
//             Xb[(i N2 + j) Kp + k] = bf16(X[i, j, k] / s_i)
//           Since s_i is a power of two, bf16(x / s_i) s_i == bf16(x): the
//           scales change no rounding. One BF16 MMA per K step, FP32 accumulate.
//   TF32x3  FP32-accurate: X is read as FP32 and every operand is split into
//           exact TF32 parts, x = x_hi + x_lo (x_hi: x rounded to TF32; x_lo:
//           x - x_hi rounded to TF32). Each K step issues two MMAs: x_hi
//           [f_hi; f_lo] (N = 2 NP, the two B parts stacked) and x_lo f_hi
//           (N = NP, into the f_lo half); the epilogue adds the two halves.
//           The dropped x_lo f_lo term and the rounding of the lo parts are
//           about 2^-22 of each product and of either sign.
//
// Pass 1, P3 = X x_3 F3^T: D[r, q] = sum_k A[r, k] B[q, k], r = (i, j), A K-major.
// Pass 2, P1 = X x_1 F1^T: D[c, a] = sum_i A[c, i] B[a, i], c = (j, k). BF16:
//   A read MN-major from Xb viewed as N1 x (N2 Kp). TF32x3: A read K-major
//   from Xt, a transposed copy of X made once per fit.
// B = F^T as operands [NP x K] (BF16: diag(s) folded into F1 for pass 2).
//
// Persistent CTAs, at most one per SM, each looping over 128-row tiles with
// warp roles:
//   warp 0        TMA producer: A tile and B slice of each K stage (a ring of as
//                 many stages as fit in shared memory, at most 8); the A tiles
//                 with an L2 evict-first hint (X is read once per pass)
//   warp 1        MMA issuer (one thread): tcgen05.mma into a double-buffered
//                 TMEM accumulator; tcgen05.commit frees stages and publishes
//                 finished accumulators
//   warps 2-5     epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//                 lanes 32 (w % 4) ..), scaled stores to global memory; with
//                 TcEpilogue::ysh also the tile's contraction with the
//                 matching factor rows (the nnTD sweep's mode-1 / mode-3 shares),
//                 by mma.sync on the tile staged in shared memory (mma32.cuh)
//   warps 6-9     TF32x3 only: split each staged A tile into x_hi (in place)
//                 and x_lo (into a 3-slot ring of its own)
// so a tile's epilogue overlaps the next tile's MMAs. The kernel is launched
// with programmatic stream serialization: the producer requests the first
// stages' A tiles (X, which no earlier kernel writes) before it waits for the
// preceding grid, and the B operands only after. Every mbarrier wait is
// bounded (about 2 s); on time-out the CTA flags an error, the other roles
// stop at their next wait, and TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <mutex>

#include "kernels.cuh"
#include "mma32.cuh"
#include "tc_ttm.cuh"

namespace nnc {
namespace tc {
namespace {

constexpr int kTileBytes = 128 * 128;  // one A stage: 128 rows x 128 bytes of K
constexpr int kThreadsTc = 320;        // 10 warps
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity`. False when the limit ran out or another role
// of this CTA has already failed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* fail,
                                          long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;  // the common case: no clock read
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*fail) return false;
    if (clock64() - t0 > limit) {
      atomicExch(const_cast<int*>(fail), 1);
      return false;
    }
  }
  return true;
}

// An L2 policy that makes lines evicted first: the A tiles of a pass (X, its
// copies) are read once, so they should not push out the data the kernels
// after the pass read again (the pass result, the shares, factors and core).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* tm, int x, int y,
                                                 uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: 128-byte swizzle, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor, FP32 accumulator, M = 128, N = n, B K-major.
// Operand format 1 = BF16 (kind::f16), 2 = TF32 (kind::tf32).
template <int KIND, bool kMN>
__device__ __forceinline__ uint32_t instr_desc(int n) {
  constexpr uint32_t fmt = KIND == kKindBf16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((kMN ? 1u : 0u) << 15) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                    uint32_t idesc, uint32_t accumulate) {
  if constexpr (KIND == kKindBf16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x_hi: x rounded to TF32 (10 stored mantissa bits), to nearest with ties away
// from zero, by the integer rule of tf32_lo below. x - x_hi is then exact in
// FP32 and takes either sign, so on nonnegative data the dropped x_lo f_lo
// terms average out; with x_hi truncated every x_lo, and every dropped term,
// would be nonnegative and the products biased low. Finite |x| below
// (2 - 2^-11) 2^127.
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// The remainder x - x_hi rounded to TF32, to nearest with ties away from zero:
// adding half of the dropped 13-bit field to the sign-magnitude bits and
// clearing the field rounds the magnitude (a carry moves into the exponent,
// as it should). Finite inputs only; this is the inner loop of the split, where
// integer operations run at full rate.
__device__ __forceinline__ float tf32_lo(float x, float hi) {
  return __uint_as_float((__float_as_uint(x - hi) + 0x1000u) & 0xFFFFE000u);
}

template <int KIND, int NP, bool FUSE = false>
struct TcLayout {
  static constexpr bool kTf32 = KIND == kKindTf32x3;
  // TF32x3: K stages rotate over kAcc accumulators that the epilogue adds in
  // FP32. The tensor core rounds its FP32 accumulation toward zero once per
  // MMA; shorter chains shrink that bias by kAcc.
  static constexpr int kAcc = kTf32 ? 128 / NP : 1;
  static_assert((kAcc & (kAcc - 1)) == 0, "accumulator index is taken by a mask");
  // TF32x3 accumulators are 2 NP columns wide: [0, NP) collects the main term
  // x_hi f_hi, [NP, 2 NP) the small terms x_hi f_lo (the same MMA of N = 2 NP
  // against the stacked [f_hi; f_lo] operand) and x_lo f_hi (an MMA of N = NP).
  static constexpr int kAccCols = kTf32 ? 2 * NP : NP;
  static constexpr int kTmemCols = 2 * kAcc * kAccCols;  // double-buffered
  static constexpr int kKStage = kTf32 ? 32 : 64;        // K elements per stage (128 bytes)
  static constexpr int kBBytes = NP * 128;               // one B slice
  // One ring stage: A | B (| B_lo right after B, so [B; B_lo] is one operand).
  static constexpr int kStageBytes = kTileBytes + kBBytes * (kTf32 ? 2 : 1);
  static constexpr int kOffB = kTileBytes;
  // TF32x3: x_lo tiles live in a short ring of their own; it only has to cover
  // the time from the split to the MMAs that read it.
  static constexpr int kLoSlots = kTf32 ? 3 : 0;
  static constexpr int kLoRing = kLoSlots > 0 ? kLoSlots : 1;  // index modulus
  static constexpr int kLoBytes = kLoSlots * kTileBytes;
  // Fused mode-1 contraction (pass X x_3 F3^T only): the tile's P3 rows and
  // the matching F2 rows, 128 x 32 FP32 each.
  static constexpr int kEpiBytes = FUSE ? 2 * 128 * 32 * 4 : 0;
  // As many stages as fit in the 227 KB of shared memory a CTA may use, less
  // the static barriers and the 1 KB alignment slack (at most 8).
  static constexpr int kStagesFit =
      (227 * 1024 - 512 - 1024 - kLoBytes - kEpiBytes) / kStageBytes;
  static constexpr int kStages = kStagesFit > 8 ? 8 : kStagesFit;
  static constexpr int kOffLo = kStages * kStageBytes;
  static constexpr int kOffEpi = kOffLo + kLoBytes;
  static constexpr int kSmem = 1024 + kOffEpi + kEpiBytes;
  static_assert(kTmemCols == 32 || kTmemCols == 64 || kTmemCols == 128 || kTmemCols == 256 ||
                kTmemCols == 512, "TMEM allocation must be a power of two >= 32 columns");
  static_assert(kStageBytes % 1024 == 0, "stages must keep 1024-byte swizzle atoms aligned");
  static_assert(!FUSE || NP == 32, "the fused contraction covers m3 <= 32");
};

// AND of `ok` over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epi_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(ok ? 1u : 0u)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

template <int KIND, bool kMN, int NP, bool FUSE>
__global__ void __launch_bounds__(kThreadsTc, 1)
tc_pass_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmBlo, int nk, int64_t ntiles, TcEpilogue ep,
               int* err) {
  using L = TcLayout<KIND, NP, FUSE>;
  static_assert(!(L::kTf32 && kMN), "TF32x3 passes read A K-major");
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[L::kStages], empty[L::kStages], accfull[2], accempty[2];
  __shared__ uint64_t lofull[L::kLoRing], loempty[L::kLoRing];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;

  // 1024-byte aligned start, derived from smem_raw by pointer arithmetic so
  // that the compiler keeps every access through it in the shared space.
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* vfail = &fail;
  // The successor kernel may be scheduled now; it waits for this grid itself.
  pdl_trigger();

  if (threadIdx.x == 0) {
    for (int s = 0; s < L::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    if constexpr (L::kTf32) {
      for (int j = 0; j < L::kLoSlots; ++j) {
        mbar_init(&lofull[j], 4);
        mbar_init(&loempty[j], 1);
      }
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 4);
    }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(L::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- TMA producer ----------------------------------------------------------
    if (lane == 0) {
      // Stages this CTA runs: tiles blockIdx.x, blockIdx.x + gridDim.x, ...
      const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
      const int64_t total = my_tiles * nk;
      const uint64_t stream_once = l2_evict_first();
      auto load_a = [&](int it_, unsigned char* st, uint64_t* bar) {
        const int64_t tile = blockIdx.x + static_cast<int64_t>(it_ / nk) * gridDim.x;
        const int m0 = static_cast<int>(tile * 128);
        const int k0 = (it_ % nk) * L::kKStage;
        if (!kMN) {
          tma_load_2d_hint(st, &tmA, k0, m0, bar, stream_once);
        } else {
          // 128 columns in 128-byte pieces: 2 (BF16) or 4 (TF32) boxes.
          constexpr int pieces = L::kTf32 ? 4 : 2;
          constexpr int piece_cols = 128 / pieces;
#pragma unroll
          for (int h = 0; h < pieces; ++h)
            tma_load_2d_hint(st + h * (kTileBytes / pieces), &tmA, m0 + h * piece_cols, k0, bar,
                             stream_once);
        }
      };
      auto load_b = [&](int it_, unsigned char* st, uint64_t* bar) {
        const int k0 = (it_ % nk) * L::kKStage;
        tma_load_2d(st + L::kOffB, &tmB, k0, 0, bar);
        if constexpr (L::kTf32) tma_load_2d(st + L::kOffB + L::kBBytes, &tmBlo, k0, 0, bar);
      };
      // X does not depend on earlier kernels: the first stages' A tiles are
      // requested before waiting for the predecessor grid, whose results (the
      // factor operands in B) are read only after the wait.
      const int pre = static_cast<int>(total < L::kStages ? total : L::kStages);
      for (int it = 0; it < pre; ++it) {
        mbar_expect_tx(&full[it], kTileBytes + L::kBBytes * (L::kTf32 ? 2 : 1));
        load_a(it, base + it * L::kStageBytes, &full[it]);
      }
      pdl_wait();
      for (int it = 0; it < pre; ++it) load_b(it, base + it * L::kStageBytes, &full[it]);
      int it = pre;
      bool ok = true;
      for (; it < total; ++it) {
        const int s = it % L::kStages;
        if (!mbar_wait(&empty[s], ((it / L::kStages) - 1) & 1, vfail)) {
          ok = false;
          break;
        }
        unsigned char* st = base + s * L::kStageBytes;
        mbar_expect_tx(&full[s], kTileBytes + L::kBBytes * (L::kTf32 ? 2 : 1));
        load_a(it, st, &full[s]);
        load_b(it, st, &full[s]);
      }
      if (!ok) {
        // Let the copies this CTA started land before it can exit (bounded).
        for (int back = 1; back <= L::kStages && it - back >= 0; ++back) {
          const int j = it - back;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[j % L::kStages], (j / L::kStages) & 1) &&
                 clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer --------------------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = instr_desc<KIND, kMN>(NP);
      const uint32_t idesc2 = instr_desc<KIND, kMN>(2 * NP);  // TF32x3: N = 2 NP
      int it = 0, tcount = 0;
      int rs = 0, rj = 0;         // stage and x_lo slot of `it`
      uint32_t rph = 0, jph = 0;  // their phase parities
      bool ok = true;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tcount) {
        const int buf = tcount & 1;
        if (tcount >= 2 && !mbar_wait(&accempty[buf], ((tcount >> 1) - 1) & 1, vfail)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t acc0 = tmem + buf * L::kAcc * L::kAccCols;
        // One thread issues every MMA, so its own instruction count per stage
        // bounds the stage rate: ring positions advance by counters, and the
        // descriptors of a stage are formed once and stepped by constants (the
        // 14-bit address field of a shared-memory descriptor counts 16 bytes).
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const uint32_t acc = acc0 + (kc & (L::kAcc - 1)) * L::kAccCols;
          if (!mbar_wait(&full[rs], rph, vfail) ||
              (L::kTf32 && !mbar_wait(&lofull[rj], jph, vfail))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + rs * L::kStageBytes);
          const uint64_t bdesc0 = smem_desc(st + L::kOffB, 16, 1024);
          uint64_t adesc0;
          if constexpr (kMN) {
            constexpr uint32_t lbo = L::kTf32 ? kTileBytes / 4 : kTileBytes / 2;
            adesc0 = smem_desc(st, lbo, 1024);
          } else {
            adesc0 = smem_desc(st, 16, 1024);
          }
          const uint64_t lodesc0 = smem_desc(smem_u32(base + L::kOffLo + rj * kTileBytes), 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // K-major: +32 bytes per K step inside the swizzled 128-byte rows.
            // MN-major: +K-step rows of 128 bytes; column pieces LBO apart.
            constexpr uint32_t astep = kMN ? (L::kTf32 ? 1024 : 2048) : 32;
            const uint64_t adesc = adesc0 + (uint64_t)((kk * astep) >> 4);
            const uint64_t bdesc = bdesc0 + (uint64_t)((kk * 32) >> 4);
            const uint32_t accum = (kc >= L::kAcc || kk != 0) ? 1u : 0u;
            if constexpr (L::kTf32) {
              // x_hi [f_hi; f_lo] into columns [0, 2 NP), then x_lo f_hi into
              // [NP, 2 NP): the accumulator of the main term x_hi f_hi gets one
              // truncating add per K step, the small terms share the other.
              mma<KIND>(acc, adesc, bdesc, idesc2, accum);
              mma<KIND>(acc + NP, lodesc0 + (uint64_t)((kk * 32) >> 4), bdesc, idesc, 1u);
            } else {
              mma<KIND>(acc, adesc, bdesc, idesc, accum);
            }
          }
          mma_commit(&empty[rs]);
          if constexpr (L::kTf32) mma_commit(&loempty[rj]);
          if (++rs == L::kStages) {
            rs = 0;
            rph ^= 1u;
          }
          if (++rj == L::kLoRing) {
            rj = 0;
            jph ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(&accfull[buf]);
      }
    }
  } else if (warp < 6) {
    // ---- epilogue (warps 2-5) ------------------------------------------------
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. 32 quarter + 31
    const int lr = quarter * 32 + lane;  // tile row of this thread
    float* Ps = reinterpret_cast<float*>(base + L::kOffEpi);  // FUSE: 128 x 32 pass rows
    float* Fs = Ps + 128 * 32;                                // FUSE: 128 x 32 factor rows
    // FUSE: the factor may come from the preceding grid.
    if constexpr (FUSE) pdl_wait();
    int tcount = 0;
    int64_t fs_slice = -1;  // FUSE: the j range whose F2 rows Fs holds
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
      const int buf = tcount & 1;
      if constexpr (FUSE) {
        if (tile % ep.y_nh != fs_slice) {
          // F2 rows of this tile's j range (F2 is not written during the pass),
          // loaded when the range changes (never, when the grid is a multiple of
          // the tiles per slab); the previous tile ended with a barrier.
          fs_slice = tile % ep.y_nh;
          const int64_t j = fs_slice * 128 + lr;
          const float* f = ep.yf + j * ep.yf_m;
          float fr[32];
          if ((ep.yf_m & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const float4 q = 4 * c < ep.yf_m ? *reinterpret_cast<const float4*>(f + 4 * c)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
              fr[4 * c] = q.x; fr[4 * c + 1] = q.y; fr[4 * c + 2] = q.z; fr[4 * c + 3] = q.w;
            }
          } else {
#pragma unroll
            for (int b = 0; b < 32; ++b) fr[b] = b < ep.yf_m ? f[b] : 0.f;
          }
          // Rows of 8 float4 chunks, chunk c stored at c ^ (row & 7): the
          // row-per-thread stores and the chunk reads below avoid bank conflicts.
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *reinterpret_cast<float4*>(Fs + lr * 32 + ((c ^ (lr & 7)) << 2)) =
                make_float4(fr[4 * c], fr[4 * c + 1], fr[4 * c + 2], fr[4 * c + 3]);
        }
      }
      const int64_t row = tile * 128 + lr;
      // Output row of the row-major layouts (-1: padding row, nothing stored)
      // and its scale, read before the wait so that the load is off the path.
      int64_t orow = -1;
      if (ep.p1_layout == 0) {
        if (row < ep.rows) orow = row;
      } else if (ep.p1_layout == 2) {
        const int64_t jj = row / ep.kp, k = row % ep.kp;
        if (jj < ep.n2 && k < ep.n3) orow = k * ep.n2 + jj;
      }
      const float sc = (orow >= 0 && ep.row_scale) ? ep.row_scale[orow / ep.rows_per_slice] : 1.f;
      const bool got = mbar_wait(&accfull[buf], (tcount >> 1) & 1, vfail);
      if constexpr (FUSE) {
        // All four warps take the same branch: the named barriers below need
        // every epilogue thread.
        if (!epi_all(got)) break;
      } else {
        // The warp-collective tcgen05.ld needs one decision for the whole warp.
        if (!__all_sync(0xffffffffu, got)) break;
      }
      tc_fence_after();
      const int nacc = nk < L::kAcc ? nk : L::kAcc;  // accumulators this tile wrote
      const uint32_t lanes = static_cast<uint32_t>(quarter * 32) << 16;
      const uint32_t accb = tmem + buf * L::kAcc * L::kAccCols + lanes;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(accb + c0, v);
        for (int q = 0; q < nacc; ++q) {
          if constexpr (L::kTf32) {
            uint32_t w[32];
            tmem_ld32(accb + q * L::kAccCols + NP + c0, w);  // x_hi f_lo
            if (q > 0) {
              uint32_t h[32];
              tmem_ld32(accb + q * L::kAccCols + c0, h);
#pragma unroll
              for (int t = 0; t < 32; ++t)
                w[t] = __float_as_uint(__uint_as_float(w[t]) + __uint_as_float(h[t]));
            }
#pragma unroll
            for (int t = 0; t < 32; ++t)
              v[t] = __float_as_uint(__uint_as_float(v[t]) + __uint_as_float(w[t]));
          } else if (q > 0) {
            uint32_t w[32];
            tmem_ld32(accb + q * L::kAccCols + c0, w);
#pragma unroll
            for (int t = 0; t < 32; ++t)
              v[t] = __float_as_uint(__uint_as_float(v[t]) + __uint_as_float(w[t]));
          }
        }
        if (ep.p1_layout != 1) {
          if (orow >= 0) {
            float* o = ep.out + orow * ep.q;
            if ((ep.q & 3) == 0) {
#pragma unroll
              for (int t = 0; t < 32; t += 4)
                if (c0 + t < ep.q)
                  *reinterpret_cast<float4*>(o + c0 + t) =
                      make_float4(__uint_as_float(v[t]) * sc, __uint_as_float(v[t + 1]) * sc,
                                  __uint_as_float(v[t + 2]) * sc, __uint_as_float(v[t + 3]) * sc);
            } else {
#pragma unroll
              for (int t = 0; t < 32; ++t)
                if (c0 + t < ep.q) o[c0 + t] = __uint_as_float(v[t]) * sc;
            }
          }
          if constexpr (FUSE) {
            // The stored P3 row (zero past m3) for the contraction below.
#pragma unroll
            for (int t = 0; t < 32; t += 4)
              *reinterpret_cast<float4*>(Ps + lr * 32 + (((t >> 2) ^ (lr & 7)) << 2)) =
                  make_float4(t < ep.q ? __uint_as_float(v[t]) * sc : 0.f,
                              t + 1 < ep.q ? __uint_as_float(v[t + 1]) * sc : 0.f,
                              t + 2 < ep.q ? __uint_as_float(v[t + 2]) * sc : 0.f,
                              t + 3 < ep.q ? __uint_as_float(v[t + 3]) * sc : 0.f);
          }
        } else {
          const int64_t jj = row / ep.kp, k = row % ep.kp;
          if (jj < ep.n2 && k < ep.n3) {
            float* o = ep.out + jj * ep.n3 + k;
#pragma unroll
            for (int t = 0; t < 32; ++t)
              if (c0 + t < ep.q) o[static_cast<int64_t>(c0 + t) * ep.slab] = __uint_as_float(v[t]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[buf]);
      if constexpr (FUSE) {
        // Contraction of the tile (one slab s, rows j0 .. j0 + 127):
        //   share[b, c] = sum_r F[j0 + r, b] P[(s, j0 + r), c]
        // on the tensor cores (mma32.cuh: TF32 operands beside the BF16
        // rounding of X, split TF32 in the FP32-accurate pass). The warp of
        // quarter q takes rows 32 q .. 32 q + 31 with the whole 32 x 32 share
        // (zero past m2, m3) in registers; the four partial shares are added
        // in quarter order.
        const int et = threadIdx.x - 64;  // 0 .. 127
        const int o0 = mma32::frag_off(lane, 0), o1 = mma32::frag_off(lane, 1);
        float acc[2][4][4];
        mma32::zero(acc);
        epi_sync();  // Ps and Fs complete
#pragma unroll
        for (int ks = 4 * quarter; ks < 4 * quarter + 4; ++ks)
          mma32::step<L::kTf32 ? 3 : 1>(acc, Fs + ks * 256, Ps + ks * 256, o0, o1);
        epi_sync();  // Ps is reused for the partial shares
        float* red = Ps;  // 4 x 32 x 32
        mma32::store(red + quarter * 1024, acc, lane);
        epi_sync();
        const int m2 = ep.yf_m, m3 = ep.q, n = m2 * m3;
        float* yo = ep.ysh + tile * n;
        for (int e = et; e < n; e += 128) {
          const int bb = e / m3, cc = e % m3, o = mma32::tile_index(bb, cc);
          const float y = ((red[o] + red[o + 1024]) + red[o + 2048]) + red[o + 3072];
          yo[ep.y_tr ? cc * m2 + bb : e] = y;
        }
        epi_sync();  // red and Fs are free for the next tile
      }
    }
  } else if constexpr (L::kTf32) {
    // ---- TF32 split of A (warps 6-9): A <- x_hi in place, x_lo to its ring ----
    const int ct = threadIdx.x - 192;  // 0 .. 127
    int it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int s = it % L::kStages, j = it % L::kLoRing;
        const bool got =
            mbar_wait(&full[s], (it / L::kStages) & 1, vfail) &&
            (it < L::kLoRing || mbar_wait(&loempty[j], ((it / L::kLoRing) - 1) & 1, vfail));
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        float4* a = reinterpret_cast<float4*>(base + s * L::kStageBytes);
        float4* alo = reinterpret_cast<float4*>(base + L::kOffLo + j * kTileBytes);
        // All loads of the stage are issued before the first store, so their
        // shared-memory latencies overlap instead of adding up.
        constexpr int kPer = kTileBytes / 16 / 128;
        float4 x[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) x[i] = a[ct + 128 * i];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          float4 h, l;
          h.x = tf32_hi(x[i].x); l.x = tf32_lo(x[i].x, h.x);
          h.y = tf32_hi(x[i].y); l.y = tf32_lo(x[i].y, h.y);
          h.z = tf32_hi(x[i].z); l.z = tf32_lo(x[i].z, h.z);
          h.w = tf32_hi(x[i].w); l.w = tf32_lo(x[i].w, h.w);
          a[ct + 128 * i] = h;
          alo[ct + 128 * i] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&lofull[j]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && fail) atomicExch(err, 1);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(L::kTmemCols)
                 : "memory");
  }
}

// ---- conversions -------------------------------------------------------------

// s_i = 2^e with max_{j,k} X[i, j, k] = f 2^e, f in [0.5, 1); 1 for an all-zero slice.
__global__ void slice_scale_kernel(const float* __restrict__ X, int64_t slab, float* scale,
                                   float* inv_scale) {
  __shared__ float red[32];
  float mx = 0.f;
  const float* x = X + static_cast<int64_t>(blockIdx.x) * slab;
  for (int64_t e = threadIdx.x; e < slab; e += blockDim.x) mx = fmaxf(mx, fabsf(x[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) {
      int e = 0;
      if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
      scale[blockIdx.x] = ldexpf(1.f, e);
      inv_scale[blockIdx.x] = ldexpf(1.f, -e);
    }
  }
}

__global__ void x_to_bf16_kernel(const float* __restrict__ X, int64_t rows, int n3, int kp,
                                 int rows_per_slice, const float* __restrict__ inv_scale,
                                 __nv_bfloat16* __restrict__ Xb) {
  const int64_t n = rows * kp;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / kp;
    const int k = static_cast<int>(e % kp);
    const float v = k < n3 ? X[r * n3 + k] * inv_scale[r / rows_per_slice] : 0.f;
    Xb[e] = __float2bfloat16_rn(v);
  }
}

// B operands of a factor F (n x m): Bt[q, k] = F[k, q] * (scale ? scale[k] : 1)
// as BF16 (bt16), or as the TF32 pair (bhi, blo); zero outside q < m, k < n.
__global__ void factor_b_kernel(const float* __restrict__ F, int n, int m, int kpad, int np,
                                const float* __restrict__ scale, __nv_bfloat16* __restrict__ bt16,
                                float* __restrict__ bhi, float* __restrict__ blo) {
  const int64_t tot = static_cast<int64_t>(np) * kpad;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < tot;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(e / kpad), k = static_cast<int>(e % kpad);
    float v = 0.f;
    if (q < m && k < n) v = F[static_cast<int64_t>(k) * m + q] * (scale ? scale[k] : 1.f);
    if (bt16) bt16[e] = __float2bfloat16_rn(v);
    if (bhi) {
      const float h = tf32_hi(v);
      bhi[e] = h;
      blo[e] = tf32_lo(v, h);
    }
  }
}

// Xt[c, i] = X[i, c] (X viewed N1 x C, Xt row length ldt >= N1, zero padded).
__global__ void transpose_kernel(const float* __restrict__ X, int64_t N1, int64_t C, int64_t ldt,
                                 float* __restrict__ Xt) {
  __shared__ float tile[32][33];
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32, i0 = static_cast<int64_t>(blockIdx.y) * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < N1 && c < C) ? X[i * C + c] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t c = c0 + r, i = i0 + threadIdx.x;
    if (c < C && i < ldt) Xt[c * ldt + i] = tile[threadIdx.x][r];
  }
}

// Xt[(k N2 + j) ldt + i] = X[i, j, k] (Xt rows (k, j), row length ldt >= N1,
// zero padded); block (k tile, i tile) of 32 x 32, looping over j.
__global__ void transpose_kj_kernel(const float* __restrict__ X, int64_t N1, int64_t N2,
                                    int64_t N3, int64_t ldt, float* __restrict__ Xt) {
  __shared__ float tile[32][33];
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * 32, i0 = static_cast<int64_t>(blockIdx.y) * 32;
  for (int64_t j = blockIdx.z; j < N2; j += gridDim.z) {
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t i = i0 + r, k = k0 + threadIdx.x;
      tile[r][threadIdx.x] = (i < N1 && k < N3) ? X[(i * N2 + j) * N3 + k] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t k = k0 + r, i = i0 + threadIdx.x;
      if (k < N3 && i < ldt) Xt[(k * N2 + j) * ldt + i] = tile[threadIdx.x][r];
    }
    __syncthreads();
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int make_map(CUtensorMap* tm, CUtensorMapDataType dt, const void* base, uint64_t inner,
             uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) {
    set_error_detail_text("cuTensorMapEncodeTiled is not available from the driver");
    return NNC_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof(buf), "cuTensorMapEncodeTiled failed (%d): dims %llu x %llu, box %u x %u",
             static_cast<int>(r), (unsigned long long)inner, (unsigned long long)outer, box_inner,
             box_outer);
    set_error_detail_text(buf);
    return NNC_ERR_CUDA;
  }
  return NNC_OK;
}

template <int KIND, bool kMN, int NP, bool FUSE>
int launch_pass(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& blo, int nk,
                int64_t tiles, const TcEpilogue& ep, int* err, int reserve, cudaStream_t s) {
  constexpr int smem = TcLayout<KIND, NP, FUSE>::kSmem;
  NNC_CUDA_TRY(raise_smem_limit((const void*)tc_pass_kernel<KIND, kMN, NP, FUSE>, smem));
  // Fewest CTAs that keep the largest tile count per CTA of a grid over the
  // SMs the pass may take: the time is the same, and the SMs left over run
  // the small kernels of the sweep that the graph places beside the pass.
  // With at least 8 tiles per SM the pass leaves `reserve` SMs to them.
  const int sms = device_sm_count();
  const int avail = (tiles >= 8LL * sms && reserve > 0 && reserve < sms / 2) ? sms - reserve : sms;
  const int64_t per = ceil_div(tiles, (int64_t)avail);
  int64_t grid = ceil_div(tiles, per);
  if (FUSE && ep.y_nh > 1) {
    // A grid that is a multiple of the tiles per slab gives every CTA tiles
    // of one j range only, so it loads its factor rows once per pass.
    const int64_t up = ceil_div(grid, ep.y_nh) * ep.y_nh;
    if (up <= avail) grid = up;
    else if (avail >= ep.y_nh) grid = avail / ep.y_nh * ep.y_nh;
  }
  NNC_CUDA_TRY(launch_pdl(tc_pass_kernel<KIND, kMN, NP, FUSE>, dim3(static_cast<unsigned>(grid)),
                          dim3(kThreadsTc), smem, s, a, b, blo, nk, tiles, ep, err));
  note_launch(s);
  return NNC_OK;
}

template <int KIND, bool kMN>
int launch_np(int np, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& blo, int nk,
              int64_t tiles, const TcEpilogue& ep, int* err, int reserve, cudaStream_t s) {
  if constexpr (!kMN) {
    if (ep.ysh)
      return launch_pass<KIND, kMN, 32, true>(a, b, blo, nk, tiles, ep, err, reserve, s);
  }
  if (np == 32) return launch_pass<KIND, kMN, 32, false>(a, b, blo, nk, tiles, ep, err, reserve, s);
  return launch_pass<KIND, kMN, 64, false>(a, b, blo, nk, tiles, ep, err, reserve, s);
}

}  // namespace

int TcPlan::init(int kind_, const float* X, int64_t N1_, int64_t N2_, int64_t N3_, int m1_,
                 int m3_, Scratch& sc, cudaStream_t s, bool p1_kj_) {
  kind = kind_;
  p1_kj = p1_kj_;
  N1 = N1_;
  N2 = N2_;
  N3 = N3_;
  m1 = m1_;
  m3 = m3_;
  np1 = m1 <= 32 ? 32 : 64;
  np3 = m3 <= 32 ? 32 : 64;
  const int kstage = kind == kKindBf16 ? 64 : 32;
  // K of pass 1 is N3 (BF16: padded rows of Xb), K of pass 2 is N1.
  kp3 = kind == kKindBf16 ? static_cast<int>(ceil_div(N3, 64) * 64) : static_cast<int>(N3);
  kb3 = static_cast<int>(ceil_div(N3, kstage) * kstage);
  kp1 = static_cast<int>(ceil_div(N1, kstage) * kstage);
  if (m1 > 64 || m3 > 64 || N1 * N2 > (1LL << 31) || N2 * kp3 > (1LL << 31)) {
    set_error_detail_text("tensor-core pass: shape outside the path (m <= 64)");
    return NNC_ERR_UNSUPPORTED;
  }
  if (kind == kKindTf32x3 && (N3 % 4) != 0) {
    set_error_detail_text("tensor-core TF32 pass: N3 must be a multiple of 4");
    return NNC_ERR_UNSUPPORTED;
  }
  const int64_t rows = N1 * N2;
  NNC_TRY(sc.get(&err, 1));
  NNC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  NNC_TRY(sc.get(&scale, static_cast<size_t>(N1)));
  NNC_TRY(sc.get(&inv_scale, static_cast<size_t>(N1)));
  if (kind == kKindBf16) {
    NNC_TRY(sc.get(&Xb, static_cast<size_t>(rows * kp3)));
    NNC_TRY(sc.get(&Bt1, static_cast<size_t>(np1) * kp1));
    NNC_TRY(sc.get(&Bt3, static_cast<size_t>(np3) * kb3));
    NNC_CUDA_TRY(cudaMemsetAsync(Bt1, 0, sizeof(__nv_bfloat16) * np1 * kp1, s));
    NNC_CUDA_TRY(cudaMemsetAsync(Bt3, 0, sizeof(__nv_bfloat16) * np3 * kb3, s));
    slice_scale_kernel<<<static_cast<unsigned>(N1), 256, 0, s>>>(X, N2 * N3, scale, inv_scale);
    note_launch(s);
    const int64_t n = rows * kp3;
    const unsigned blocks =
        static_cast<unsigned>(ceil_div(n, 256) < 16384 ? ceil_div(n, 256) : 16384);
    x_to_bf16_kernel<<<blocks, 256, 0, s>>>(X, rows, static_cast<int>(N3), kp3,
                                           static_cast<int>(N2), inv_scale, Xb);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    NNC_TRY(make_map(&mapA3, bf, Xb, kp3, rows, static_cast<uint64_t>(kp3) * 2, 64, 128));
    NNC_TRY(make_map(&mapB3, bf, Bt3, kb3, np3, static_cast<uint64_t>(kb3) * 2, 64, np3));
    NNC_TRY(make_map(&mapA1, bf, Xb, static_cast<uint64_t>(N2) * kp3, N1,
                     static_cast<uint64_t>(N2) * kp3 * 2, 64, 64));
    NNC_TRY(make_map(&mapB1, bf, Bt1, kp1, np1, static_cast<uint64_t>(kp1) * 2, 64, np1));
    mapB3lo = mapB3;
    mapB1lo = mapB1;
  } else {
    NNC_TRY(sc.get(&B1hi, static_cast<size_t>(np1) * kp1));
    NNC_TRY(sc.get(&B1lo, static_cast<size_t>(np1) * kp1));
    NNC_TRY(sc.get(&B3hi, static_cast<size_t>(np3) * kb3));
    NNC_TRY(sc.get(&B3lo, static_cast<size_t>(np3) * kb3));
    NNC_CUDA_TRY(cudaMemsetAsync(B1hi, 0, sizeof(float) * np1 * kp1, s));
    NNC_CUDA_TRY(cudaMemsetAsync(B1lo, 0, sizeof(float) * np1 * kp1, s));
    NNC_CUDA_TRY(cudaMemsetAsync(B3hi, 0, sizeof(float) * np3 * kb3, s));
    NNC_CUDA_TRY(cudaMemsetAsync(B3lo, 0, sizeof(float) * np3 * kb3, s));
    scale = nullptr;
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    NNC_TRY(make_map(&mapA3, f32, X, N3, rows, static_cast<uint64_t>(N3) * 4, 32, 128));
    NNC_TRY(make_map(&mapB3, f32, B3hi, kb3, np3, static_cast<uint64_t>(kb3) * 4, 32, np3));
    NNC_TRY(make_map(&mapB3lo, f32, B3lo, kb3, np3, static_cast<uint64_t>(kb3) * 4, 32, np3));
    // Pass 2 reads Xt = X viewed (N1 x N2 N3), transposed: K-major rows of N1p
    // in the order (j, k), or (k, j) for p1_kj.
    const int64_t C = N2 * N3, n1p = ceil_div(N1, 4) * 4;
    NNC_TRY(sc.get(&Xt, static_cast<size_t>(C * n1p)));
    if (p1_kj) {
      dim3 tgrid(static_cast<unsigned>(ceil_div(N3, 32)), static_cast<unsigned>(ceil_div(n1p, 32)),
                 static_cast<unsigned>(N2 < 65535 ? N2 : 65535));
      transpose_kj_kernel<<<tgrid, dim3(32, 8), 0, s>>>(X, N1, N2, N3, n1p, Xt);
    } else {
      dim3 tgrid(static_cast<unsigned>(ceil_div(C, 32)), static_cast<unsigned>(ceil_div(n1p, 32)));
      transpose_kernel<<<tgrid, dim3(32, 8), 0, s>>>(X, N1, C, n1p, Xt);
    }
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    NNC_TRY(make_map(&mapA1, f32, Xt, n1p, C, static_cast<uint64_t>(n1p) * 4, 32, 128));
    NNC_TRY(make_map(&mapB1, f32, B1hi, kp1, np1, static_cast<uint64_t>(kp1) * 4, 32, np1));
    NNC_TRY(make_map(&mapB1lo, f32, B1lo, kp1, np1, static_cast<uint64_t>(kp1) * 4, 32, np1));
  }
  return NNC_OK;
}

int TcPlan::convert_b3(const float* F3, cudaStream_t s) const {
  factor_b_kernel<<<64, 256, 0, s>>>(F3, static_cast<int>(N3), m3, kb3, np3, nullptr, Bt3, B3hi,
                                     B3lo);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

int TcPlan::convert_b1(const float* F1, cudaStream_t s) const {
  factor_b_kernel<<<64, 256, 0, s>>>(F1, static_cast<int>(N1), m1, kp1, np1,
                                     kind == kKindBf16 ? scale : nullptr, Bt1, B1hi, B1lo);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

bool TcPlan::y1_fusable(int m2) const {
  // Tiles of pass 1 are single (i, j0 .. j0 + 127) row blocks when N2 % 128
  // == 0; the tile contraction runs on the tensor cores, which keeps it off
  // the BF16 pass's stage rate too.
  return np3 == 32 && m2 >= 1 && m2 <= 32 && N2 % 128 == 0;
}

bool TcPlan::y3_fusable(int m2) const {
  // Tiles of pass 2 are single (k, j0 .. j0 + 127) row blocks only when read
  // from the (k, j)-ordered Xt.
  return kind == kKindTf32x3 && p1_kj && np1 == 32 && m2 >= 1 && m2 <= 32 && N2 % 128 == 0;
}

int TcPlan::pass3(const float* F3, float* P3, cudaStream_t s, bool convert, const float* F2,
                  int m2, float* Y1) const {
  if (convert) NNC_TRY(convert_b3(F3, s));
  TcEpilogue ep{};
  ep.out = P3;
  ep.q = m3;
  ep.rows = N1 * N2;
  ep.rows_per_slice = N2;
  ep.row_scale = kind == kKindBf16 ? scale : nullptr;
  if (Y1) {
    if (!F2 || !y1_fusable(m2)) return NNC_ERR_UNSUPPORTED;
    ep.ysh = Y1;
    ep.yf = F2;
    ep.yf_m = m2;
    ep.y_nh = N2 / 128;
  }
  const int64_t tiles = ceil_div(N1 * N2, 128);
  const int stagek = kind == kKindBf16 ? 64 : 32;
  const int nk = static_cast<int>(ceil_div(N3, stagek));
  if (kind == kKindBf16)
    return launch_np<kKindBf16, false>(np3, mapA3, mapB3, mapB3lo, nk, tiles, ep, err,
                                       reserve_sms, s);
  return launch_np<kKindTf32x3, false>(np3, mapA3, mapB3, mapB3lo, nk, tiles, ep, err,
                                       reserve_sms, s);
}

int TcPlan::pass1(const float* F1, float* P1, cudaStream_t s, bool convert, const float* F2,
                  int m2, float* Y3) const {
  if (convert) NNC_TRY(convert_b1(F1, s));
  TcEpilogue ep{};
  ep.out = P1;
  ep.q = m1;
  ep.kp = kp3;
  ep.n2 = N2;
  ep.n3 = N3;
  ep.slab = N2 * N3;
  if (!p1_kj) {
    ep.p1_layout = 1;
  } else if (kind == kKindBf16) {
    ep.p1_layout = 2;  // MN-major tiles of Xb have rows (j, k)
  } else {
    ep.p1_layout = 0;  // Xt already has rows (k, j)
    ep.rows = N2 * N3;
  }
  if (Y3) {
    if (!F2 || !y3_fusable(m2)) return NNC_ERR_UNSUPPORTED;
    ep.ysh = Y3;
    ep.yf = F2;
    ep.yf_m = m2;
    ep.y_tr = 1;  // Y3[k] is stored m1 x m2
    ep.y_nh = N2 / 128;
  }
  const int64_t tiles = ceil_div(N2 * kp3, 128);
  const int stagek = kind == kKindBf16 ? 64 : 32;
  const int nk = static_cast<int>(ceil_div(N1, stagek));
  if (kind == kKindBf16)
    return launch_np<kKindBf16, true>(np1, mapA1, mapB1, mapB1lo, nk, tiles, ep, err,
                                      reserve_sms, s);
  return launch_np<kKindTf32x3, false>(np1, mapA1, mapB1, mapB1lo, nk, tiles, ep, err,
                                       reserve_sms, s);
}

// Self-test of the bounded waits: one CTA waits, with a limit of `cycles`, on
// the first phase of an mbarrier that expects one arrival and gets none (no
// copy or MMA is in flight). The wait must give up and flag the failure the
// way the pass kernel's roles do; status[0] = 1 then, 0 if the wait returned.
__global__ void wait_selftest_kernel(long long cycles, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int fail;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool got = mbar_wait(&bar, 0, &fail, cycles);
  __syncthreads();
  if (threadIdx.x == 0) status[0] = (got && !fail) ? 0 : 1;
}

int wait_selftest(long long cycles, cudaStream_t s) {
  if (cycles < 0) return NNC_ERR_INVALID_ARG;
  Scratch sc(s);
  int* d = nullptr;
  NNC_TRY(sc.get(&d, 1));
  NNC_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(int), s));
  wait_selftest_kernel<<<1, 32, 0, s>>>(cycles, d);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  int h = 0;
  NNC_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    set_error_detail_text("self-test: the bounded wait gave up as it should");
    return NNC_ERR_TIMEOUT;
  }
  return NNC_OK;
}

int TcPlan::check(cudaStream_t s) const {
  int h = 0;
  NNC_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NNC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    set_error_detail_text("tensor-core mode product: a pipeline wait timed out");
    return NNC_ERR_TIMEOUT;
  }
  return NNC_OK;
}

}  // namespace tc
}  // namespace nnc
