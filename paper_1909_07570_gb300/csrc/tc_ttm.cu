// Tensor-core (tcgen05) mode products for the BF16 path: the two passes over X
// of an nnTD sweep (n-mode multiplication, Appendix A).
//
// X is kept as a BF16 copy Xb with per-slice power-of-two scales s_i (mode-1
// slices) and rows padded with zeros to Kp = roundup(N3, 64):
//   Xb[(i N2 + j) Kp + k] = bf16(X[i, j, k] / s_i)            (k < N3)
// Because s_i is a power of two, bf16(x / s_i) * s_i == bf16(x): the scaling
// changes no rounding and only keeps slices of very different magnitude in
// range.
//
// Pass 1, P3 = X x_3 F3^T: D[r, q] = sum_k Xb[r, k] Bt3[q, k] with r = (i, j),
//   A = Xb tile (128 rows x 64 k, K-major), B = Bt3 = bf16(F3^T) (NP x Kp);
//   the epilogue multiplies row r by s_i.
// Pass 2, P1 = X x_1 F1^T: D[c, a] = sum_i Xb[i, c] Bt1[a, i] with c = (j, k),
//   A = Xb viewed as N1 x (N2 Kp) read MN-major (128 columns x 64 i),
//   B = Bt1 = bf16(diag(s) F1)^T, so the scales ride on F1.
//
// One CTA computes one 128-row tile with a single tcgen05.mma accumulator of
// NP (32 or 64) FP32 columns in tensor memory:
//   warp 0 / lane 0  TMA producer: all of B once, then A through a 4-stage ring
//   warp 1 / lane 0  MMA issuer: 4 MMAs (K = 16 each) per stage, tcgen05.commit
//                    frees the stage; a final commit signals the accumulator
//   all 4 warps      epilogue: tcgen05.ld (warp w owns TMEM lanes 32w..32w+31)
// Shared-memory tiles use the 128-byte swizzle that TMA writes and the MMA
// descriptors read. Every mbarrier wait is bounded; on time-out the CTA
// records an error, waits (bounded) for its own copies and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <mutex>

#include "kernels.cuh"
#include "tc_ttm.cuh"

namespace nnc {
namespace tc {
namespace {

constexpr int kStages = 4;
constexpr int kStageBytes = 128 * 64 * 2;  // one A tile: 128 x 64 bf16
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

// Bounded wait on phase `parity`; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
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

// Shared-memory matrix descriptor: 128-byte swizzle, leading / stride byte
// offsets as given, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, M = 128, N = NP,
// B K-major, A K-major or MN-major.
template <bool kMN, int NP>
__device__ __forceinline__ uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((kMN ? 1u : 0u) << 15) |
         (static_cast<uint32_t>(NP >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
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

template <bool kMN, int NP>
__global__ void __launch_bounds__(128, 1)
ttm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int nk, TcEpilogue ep, int* err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bars[2 * kStages + 2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;

  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* sA = base;                        // kStages x 16 KB
  unsigned char* sB = base + kStages * kStageBytes;  // nk x NP x 128 B
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* bfull = bars + 2 * kStages;
  uint64_t* accfull = bars + 2 * kStages + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * 128;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bfull, 1);
    mbar_init(accfull, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(NP)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer --------------------------------------------------------
    mbar_expect_tx(bfull, static_cast<uint32_t>(nk) * NP * 128);
    for (int c = 0; c < nk; ++c) tma_load_2d(sB + c * NP * 128, &tmB, c * 64, 0, bfull);
    int issued = 0;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kStages;
      if (kc >= kStages && !mbar_wait(&empty[s], ((kc / kStages) - 1) & 1)) {
        atomicExch(&fail, 1);
        break;
      }
      mbar_expect_tx(&full[s], kStageBytes);
      if (!kMN) {
        tma_load_2d(sA + s * kStageBytes, &tmA, kc * 64, static_cast<int>(m0), &full[s]);
      } else {
        tma_load_2d(sA + s * kStageBytes, &tmA, static_cast<int>(m0), kc * 64, &full[s]);
        tma_load_2d(sA + s * kStageBytes + kStageBytes / 2, &tmA, static_cast<int>(m0) + 64,
                    kc * 64, &full[s]);
      }
      issued = kc + 1;
    }
    if (fail) {
      // Let this CTA's copies land before the CTA can exit.
      mbar_wait(bfull, 0);
      for (int kc = (issued > kStages ? issued - kStages : 0); kc < issued; ++kc)
        mbar_wait(&full[kc % kStages], (kc / kStages) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----------------------------------------------------------
    const uint32_t idesc = instr_desc<kMN, NP>();
    bool ok = mbar_wait(bfull, 0);
    for (int kc = 0; ok && kc < nk; ++kc) {
      const int s = kc % kStages;
      if (!mbar_wait(&full[s], (kc / kStages) & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * kStageBytes);
      const uint32_t b0 = smem_u32(sB + kc * NP * 128);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        // K-major A: +32 B per K = 16 inside the swizzled 128 B row.
        // MN-major A: +16 rows of 128 B per K = 16; the two 64-column halves
        // of the tile are kStageBytes / 2 apart (leading byte offset).
        const uint64_t adesc = kMN ? smem_desc(a0 + kk * 2048, kStageBytes / 2, 1024)
                                   : smem_desc(a0 + kk * 32, 16, 1024);
        const uint64_t bdesc = smem_desc(b0 + kk * 32, 16, 1024);
        mma_bf16(tmem, adesc, bdesc, idesc, (kc | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    if (!ok) atomicExch(&fail, 1);
    mma_commit(accfull);  // fires once every MMA issued above has completed
  }
  __syncwarp();

  // ---- epilogue: TMEM -> registers -> global ---------------------------------
  const bool have = mbar_wait(accfull, 0);
  tc_fence_after();
  if (!have) atomicExch(&fail, 1);
  __syncthreads();
  if (!fail) {
    const int64_t row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      if (!kMN) {
        if (row < ep.rows) {
          const float sc = ep.row_scale[row / ep.rows_per_slice];
          float* o = ep.out + row * ep.q;
#pragma unroll
          for (int t = 0; t < 32; ++t)
            if (c0 + t < ep.q) o[c0 + t] = __uint_as_float(v[t]) * sc;
        }
      } else {
        const int64_t j = row / ep.kp, k = row % ep.kp;
        if (j < ep.n2 && k < ep.n3) {
          float* o = ep.out + j * ep.n3 + k;
#pragma unroll
          for (int t = 0; t < 32; ++t)
            if (c0 + t < ep.q) o[static_cast<int64_t>(c0 + t) * ep.slab] = __uint_as_float(v[t]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && fail) atomicExch(err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NP)
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

// Bt[q, k] = bf16(F[k, q] * (scale ? scale[k] : 1)), zero outside q < m, k < n.
__global__ void factor_bt_kernel(const float* __restrict__ F, int n, int m, int kpad, int np,
                                 const float* __restrict__ scale, __nv_bfloat16* __restrict__ Bt) {
  const int64_t tot = static_cast<int64_t>(np) * kpad;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < tot;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(e / kpad), k = static_cast<int>(e % kpad);
    float v = 0.f;
    if (q < m && k < n) v = F[static_cast<int64_t>(k) * m + q] * (scale ? scale[k] : 1.f);
    Bt[e] = __float2bfloat16_rn(v);
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

int make_map(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer,
             uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr) {
    set_error_detail_text("cuTensorMapEncodeTiled is not available from the driver");
    return NNC_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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

size_t smem_bytes(int nk, int np) {
  return 1024 + static_cast<size_t>(kStages) * kStageBytes + static_cast<size_t>(nk) * np * 128;
}

template <bool kMN, int NP>
int launch_pass(const CUtensorMap& a, const CUtensorMap& b, int nk, int64_t tiles,
                const TcEpilogue& ep, int* err, cudaStream_t s) {
  const size_t smem = smem_bytes(nk, NP);
  NNC_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<kMN, NP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  ttm_tc_kernel<kMN, NP><<<static_cast<unsigned>(tiles), 128, smem, s>>>(a, b, nk, ep, err);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

}  // namespace

int TcPlan::init(const float* X, int64_t N1_, int64_t N2_, int64_t N3_, int m1_, int m3_,
                 Scratch& sc, cudaStream_t s) {
  N1 = N1_;
  N2 = N2_;
  N3 = N3_;
  m1 = m1_;
  m3 = m3_;
  kp3 = static_cast<int>(ceil_div(N3, 64) * 64);
  kp1 = static_cast<int>(ceil_div(N1, 64) * 64);
  np1 = m1 <= 32 ? 32 : 64;
  np3 = m3 <= 32 ? 32 : 64;
  if (m1 > 64 || m3 > 64 || smem_bytes(kp3 / 64, np3) > 220 * 1024 ||
      smem_bytes(kp1 / 64, np1) > 220 * 1024 || N1 * N2 > (1LL << 31) ||
      N2 * kp3 > (1LL << 31)) {
    set_error_detail_text("NNC_BF16_REFINE: shape outside the tensor-core path (m <= 64, "
                          "N1 and N3 <= 1600)");
    return NNC_ERR_UNSUPPORTED;
  }
  const int64_t rows = N1 * N2;
  NNC_TRY(sc.get(&Xb, static_cast<size_t>(rows * kp3)));
  NNC_TRY(sc.get(&scale, static_cast<size_t>(N1)));
  NNC_TRY(sc.get(&inv_scale, static_cast<size_t>(N1)));
  NNC_TRY(sc.get(&Bt1, static_cast<size_t>(np1) * kp1));
  NNC_TRY(sc.get(&Bt3, static_cast<size_t>(np3) * kp3));
  NNC_TRY(sc.get(&err, 1));
  NNC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  NNC_CUDA_TRY(cudaMemsetAsync(Bt1, 0, sizeof(__nv_bfloat16) * np1 * kp1, s));
  NNC_CUDA_TRY(cudaMemsetAsync(Bt3, 0, sizeof(__nv_bfloat16) * np3 * kp3, s));
  slice_scale_kernel<<<static_cast<unsigned>(N1), 256, 0, s>>>(X, N2 * N3, scale, inv_scale);
  note_launch(s);
  const int64_t n = rows * kp3;
  const unsigned blocks = static_cast<unsigned>(ceil_div(n, 256) < 16384 ? ceil_div(n, 256) : 16384);
  x_to_bf16_kernel<<<blocks, 256, 0, s>>>(X, rows, static_cast<int>(N3), kp3,
                                         static_cast<int>(N2), inv_scale, Xb);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  NNC_TRY(make_map(&mapA3, Xb, kp3, rows, static_cast<uint64_t>(kp3) * 2, 64, 128));
  NNC_TRY(make_map(&mapB3, Bt3, kp3, np3, static_cast<uint64_t>(kp3) * 2, 64, np3));
  NNC_TRY(make_map(&mapA1, Xb, static_cast<uint64_t>(N2) * kp3, N1,
                   static_cast<uint64_t>(N2) * kp3 * 2, 64, 64));
  NNC_TRY(make_map(&mapB1, Bt1, kp1, np1, static_cast<uint64_t>(kp1) * 2, 64, np1));
  return NNC_OK;
}

int TcPlan::pass3(const float* F3, float* P3, cudaStream_t s, bool convert) const {
  if (convert) {
    factor_bt_kernel<<<64, 256, 0, s>>>(F3, static_cast<int>(N3), m3, kp3, np3, nullptr, Bt3);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
  }
  TcEpilogue ep{};
  ep.out = P3;
  ep.q = m3;
  ep.rows = N1 * N2;
  ep.rows_per_slice = N2;
  ep.row_scale = scale;
  const int64_t tiles = ceil_div(N1 * N2, 128);
  if (np3 == 32) return launch_pass<false, 32>(mapA3, mapB3, kp3 / 64, tiles, ep, err, s);
  return launch_pass<false, 64>(mapA3, mapB3, kp3 / 64, tiles, ep, err, s);
}

int TcPlan::pass1(const float* F1, float* P1, cudaStream_t s, bool convert) const {
  if (convert) {
    factor_bt_kernel<<<64, 256, 0, s>>>(F1, static_cast<int>(N1), m1, kp1, np1, scale, Bt1);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
  }
  TcEpilogue ep{};
  ep.out = P1;
  ep.q = m1;
  ep.kp = kp3;
  ep.n2 = N2;
  ep.n3 = N3;
  ep.slab = N2 * N3;
  const int64_t tiles = ceil_div(N2 * kp3, 128);
  if (np1 == 32) return launch_pass<true, 32>(mapA1, mapB1, kp1 / 64, tiles, ep, err, s);
  return launch_pass<true, 64>(mapA1, mapB1, kp1 / 64, tiles, ep, err, s);
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
