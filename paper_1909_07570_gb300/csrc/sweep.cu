// Fused kernels of one nnTD sweep around the two passes over X.
//
// With P3 = X x_3 F3^T ((N1 N2) x m3) and P1 = X x_1 F1^T (rows (k, j) x m1)
// from the passes, a sweep is (S_k = F_k^T F_k, Eq. unfolding:property):
//
//   update (mode 1) per slab i: Y1[i] = F2^T P3[i, :, :]           (m2 x m3)
//                               (or the sum of its shares formed by pass 1)
//                               Num1[i, a] = <Y1[i], G[a, :, :]>
//                               F1[i, :] <- MU with Den = F1[i, :] H1
//   hmat  (mode 2) per b:       S1 = F1^T F1;  W[:, b, :] = S1 G[:, b, :] S3
//                               H2[b, b'] = <W[:, b, :], G[:, b', :]>
//   update (mode 2) per row j:  Y2[:, j, :] = F1^T P3[:, j, :];  Num2 (numerator only)
//   mu_rows (mode 2):           MU on F2 with Den = F2 H2
//   hmat  (mode 3) per c:       S2 = F2^T F2;  W3 = G x_1 S1 x_2 S2 (kept);  H3
//   update (mode 3) per slab k: Y3[k] = P1[k, :, :]^T F2  (m1 x m2, kept)
//                               (or the sum of its shares formed by pass 2)
//                               Num3[k, c] = <Y3[k], G[:, :, c]>;  MU on F3
//   core_a (one block per a):   S3 = F3^T F3; M[a] = Y3[:, a, :]^T F3 (= (X x_1 F1^T x_2 F2^T x_3 F3^T)[a]);
//                               D = W3 x_3 S3;  G <- MU(G, M, D); W1 = G x_2 S2 x_3 S3
//   core_b (one block per a):   H1 = unfold_1(W1) unfold_1(G)^T for the next sweep;
//                               trace = sqrt(||X||^2 - 2<M,G> + <G, G x_k S_k>)/||X||
//                               with <G, G x_k S_k> = sum S1 .* H1^T (last block)
//
// An update runs as updt_kernel (the GEMM Y_r on the tensor cores, FP32 data
// with m <= 32), updm_kernel (the GEMM on the SIMT pipes) or upds_kernel (Y_r
// from the pass's shares), two rows per block; all three end in the same
// numerators and MU step. The other kernels are latency-bound (a few MFLOP
// each on L2-resident data), so each block requests everything it needs up
// front (cp.async) and spreads every contraction over all its threads: the
// block GEMM splits the contraction across thread groups (4 x 4 register
// tiles per thread). Most blocks run
// their code once per sweep with a cold instruction cache, so the shared
// helpers are kept out of line and not unrolled (one copy of the code per
// kernel). Every reduction runs in a fixed order, so results are
// deterministic. The BF16 path also writes, from the mode-1 and mode-3
// updates, the BF16 operand of the next pass over X.
#include <cuda_bf16.h>

#include <type_traits>

#include "kernels.cuh"
#include "mma32.cuh"
#include "sweep.cuh"
#include "tma.cuh"

namespace nnc {
namespace {

constexpr int kThreads = 256;
constexpr int KC = 32;  // contraction chunk staged in shared memory

__host__ __device__ constexpr int r4(int x) { return (x + 3) & ~3; }
// Shared-memory regions start on 4-element boundaries so that the 4-wide loads
// (float4 / 2 x double2) stay 16-byte aligned.
__host__ __device__ constexpr size_t al4(size_t x) { return (x + 3) & ~static_cast<size_t>(3); }

// Writes the tensor-core operand entry of a new factor value (see UpdArgs).
template <typename T>
__device__ __forceinline__ void write_operand(const UpdArgs<T>& a, int64_t r, int v, T nv) {
  if constexpr (std::is_same<T, float>::value) {
    const float x = nv * (a.bt_scale ? a.bt_scale[r] : 1.f);
    const int64_t idx = (int64_t)v * a.bt_ld + r;
    if (a.bt) a.bt[idx] = __float2bfloat16_rn(x);
    if (a.bhi) {
      // x rounded to TF32, and the remainder rounded to TF32, both to nearest
      // with ties away from zero (the pass kernel's rule for its operand splits).
      const float h = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
      a.bhi[idx] = h;
      a.blo[idx] = __uint_as_float((__float_as_uint(x - h) + 0x1000u) & 0xFFFFE000u);
    }
  }
}

template <typename T>
__device__ __forceinline__ T mu_step(T theta, T num, T den, T eps) {
  const T v = theta * num / (den > eps ? den : eps);
  return v > T(0) ? v : T(0);
}

// Stages rows [0, nrows) x cols [0, ncols) of a tile into shared memory:
// dst[r * lds + c] = src[r * ldg + c] for r < vrows and c < vcols, else 0.
// ncols and lds are multiples of 4. With vec (src and ldg 16-byte aligned)
// whole 16-byte vectors are copied; otherwise single elements. Indices advance
// by increments, without divisions in the loop.
template <typename T>
__device__ __forceinline__ void stage_tile(T* dst, int lds, const T* __restrict__ src, int64_t ldg,
                                           int nrows, int ncols, int vrows, int vcols, bool vec) {
  if (vec) {
    constexpr int W = 16 / (int)sizeof(T);
    const int vpr = ncols / W;  // vectors per row
    const int total = nrows * vpr;
    const int step = blockDim.x;
    int r = threadIdx.x / vpr, cv = threadIdx.x % vpr;
    const int dr = step / vpr, dc = step % vpr;
    for (int v = threadIdx.x; v < total; v += step) {
      const int c = cv * W;
      int valid = (r < vrows) ? vcols - c : 0;
      valid = valid < 0 ? 0 : (valid > W ? W : valid);
      cp_vec(dst + r * lds + c, valid ? src + (int64_t)r * ldg + c : src, valid);
      r += dr;
      cv += dc;
      if (cv >= vpr) {
        cv -= vpr;
        ++r;
      }
    }
  } else {
    const int total = nrows * ncols;
    const int step = blockDim.x;
    int r = threadIdx.x / ncols, c = threadIdx.x % ncols;
    const int dr = step / ncols, dc = step % ncols;
    for (int e = threadIdx.x; e < total; e += step) {
      const bool ok = r < vrows && c < vcols;
      cp_elem(dst + r * lds + c, ok ? src + (int64_t)r * ldg + c : src, ok);
      r += dr;
      c += dc;
      if (c >= ncols) {
        c -= ncols;
        ++r;
      }
    }
  }
}

__device__ __forceinline__ bool aligned16(const void* p, int64_t ld_elems, int elem) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && (((ld_elems * elem) & 15) == 0);
}

// ---- 4-wide shared-memory loads (16-byte aligned rows) ----------------------
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T>
__device__ __forceinline__ void zero4x4(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}

// dst[e] = src[e] for e < n by cp.async (16-byte vectors when both ends allow),
// issued by the whole block; the caller commits and waits.
template <typename T>
__device__ __noinline__ void cp_flat(T* dst, const T* __restrict__ src, int64_t n) {
  constexpr int W = 16 / (int)sizeof(T);
  if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int64_t nv = n / W;
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) cp_vec(dst + v * W, src + v * W, W);
    for (int64_t e = nv * W + threadIdx.x; e < n; e += blockDim.x) cp_elem(dst + e, src + e, true);
  } else {
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) cp_elem(dst + e, src + e, true);
  }
}

// ---- block GEMM C = A^T B ----------------------------------------------------
// C[u][c] = sum_{t < len} A[t lda + u] B[t ldb + c], u < mu, c < mc (both <= 64),
// computed by one block: each thread owns a 4 x 4 tile of C for one of `groups`
// interleaved subsets of t (split-K inside the block, so every thread works
// even for small mu, mc); the partial tiles are added in group order. A and B
// are staged by cp.async in chunks of kch rows, two chunks in flight; `stage`
// holds gemm_stage_elems of the dimensions and length kch was chosen for.
__host__ __device__ inline int gemm_tiles(int mu, int mc) { return (r4(mu) / 4) * (r4(mc) / 4); }
__host__ __device__ inline int gemm_groups(int mu, int mc) {
  const int g = kThreads / gemm_tiles(mu, mc);
  return g > 1 ? g : 1;
}
// Rows per chunk: the staging buffers of A and B take at most 64 KB (FP32) or
// 24 KB (FP64) in all, chunks are a multiple of 8 rows and no longer than the
// contraction needs. A contraction of up to 256 rows (FP32, m <= 32) is staged
// in one round trip into a single buffer; a longer one is double-buffered in
// chunks of half that size, so that the staging of a block never exceeds the
// budget and several blocks stay resident per SM (at 512 rows and m = 32 the
// two 128-row buffers take 64 KB, three blocks per SM, where two 256-row
// buffers took 128 KB and one).
__host__ __device__ inline int gemm_kch(int mu, int mc, int elem, int len) {
  const int budget = elem > 4 ? 3 * 1024 : 16 * 1024;  // elements of the staging buffers
  int k = budget / (r4(mu) + r4(mc));
  k = k > 256 ? 256 : k;
  const int need = (len + 7) & ~7;
  if (need > k) k /= 2;  // two buffers share the budget
  k = k > need ? need : k;
  k &= ~7;
  return k < 8 ? 8 : k;
}
// Staging elements for gemm_tn_block with these dimensions: one buffer when a
// single chunk covers the contraction, two otherwise; at least the partial
// tiles of the group reduction (at most 16 per thread).
__host__ __device__ inline size_t gemm_stage_elems(int mu, int mc, int elem, int len) {
  const int kch = gemm_kch(mu, mc, elem, len);
  const size_t nbuf = len > kch ? 2 : 1;
  const size_t st = nbuf * kch * (r4(mu) + r4(mc));
  const size_t red = (size_t)16 * kThreads;
  return al4(st > red ? st : red);
}

template <typename T>
__device__ __noinline__ void gemm_tn_block(const T* __restrict__ A, int64_t lda, int mu,
                              const T* __restrict__ B, int64_t ldb, int mc, int len, int kch,
                              T* C, T* stage) {
  const int mu4 = r4(mu), mc4 = r4(mc), tq = mc4 / 4;
  const int tiles = gemm_tiles(mu, mc), groups = gemm_groups(mu, mc);
  const int g = threadIdx.x / tiles, t = threadIdx.x % tiles;
  const bool act = g < groups;
  const int u0 = (t / tq) * 4, c0 = (t % tq) * 4;
  // A Gram (B is A) stages its operand once.
  const bool gram = A == B && lda == ldb && mu == mc;
  T* As = stage;
  T* Bs = gram ? As : stage + (len > kch ? 2 : 1) * kch * mu4;
  const bool vecA = aligned16(A, lda, sizeof(T)), vecB = aligned16(B, ldb, sizeof(T));
  const int nch = (len + kch - 1) / kch;
  auto issue = [&](int c, int buf) {
    const int t0 = c * kch, tn = min(kch, len - t0);
    stage_tile(As + buf * kch * mu4, mu4, A + (int64_t)t0 * lda, lda, tn, mu4, tn, mu, vecA);
    if (!gram)
      stage_tile(Bs + buf * kch * mc4, mc4, B + (int64_t)t0 * ldb, ldb, tn, mc4, tn, mc, vecB);
    cp_commit();
  };
  T acc[4][4];
  zero4x4(acc);
  if (nch > 0) issue(0, 0);
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) {
      issue(c + 1, (c + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (act) {
      const int kn = min(kch, len - c * kch);
      const T* a = As + (c & 1) * kch * mu4 + u0;
      const T* b = Bs + (c & 1) * kch * mc4 + c0;
#pragma unroll 1
      for (int k = g; k < kn; k += groups) {
        T x[4], y[4];
        ld4(a + k * mu4, x);
        ld4(b + k * mc4, y);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (nch == 0) {
    cp_wait<0>();
    __syncthreads();
  }
  T* red = stage;  // the staging buffers are free after the last barrier
  if (act) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (u0 + i < mu && c0 + j < mc) red[((int64_t)g * mu + u0 + i) * mc + c0 + j] = acc[i][j];
  }
  __syncthreads();
  const int n = mu * mc;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    T v = T(0);
    for (int q = 0; q < groups; ++q) v += red[q * n + e];
    C[e] = v;
  }
  __syncthreads();
}

// C (m x n) = A (m x k) B (k x n), all row-major in shared memory; whole block.
template <typename T>
__device__ __noinline__ void smem_gemm(const T* A, const T* B, T* C, int m, int k, int n) {
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    T s0 = T(0), s1 = T(0);
    int w = 0;
    for (; w + 1 < k; w += 2) {
      s0 = fma(A[i * k + w], B[w * n + j], s0);
      s1 = fma(A[i * k + w + 1], B[(w + 1) * n + j], s1);
    }
    if (w < k) s0 = fma(A[i * k + w], B[w * n + j], s0);
    C[e] = s0 + s1;
  }
}

// out0[q] = <x0, Y[q, :]> (and out1[q] = <x1, Y[q, :]> when x1 is given) for
// q < nq: rows of length n, row stride n; x0, x1 in shared memory, Y in
// global or shared memory. NS = 8 threads (4 when nq > 32) share a row, so the
// block reads every Y row with many independent loads in flight (a warp per
// row, a few loads at a time, left the loop waiting on the latency of the
// core's reads from L2); thread s of a row takes the 4-element vectors
// s, s + NS, ... (16-byte loads when Y's rows are 16-byte aligned), and the
// NS partial sums are added by a fixed shuffle tree. Blocks that run this at
// the same time on the same Y start at different rows (row (k + blockIdx.x)
// % nq where a lone block would take row k): hundreds of blocks requesting
// the same lines of L2 at once otherwise queue behind each other. Each row's
// arithmetic is the same either way.
template <typename T>
__device__ __noinline__ void rows_dot2(const T* x0, const T* x1, const T* Y, int n, int nq,
                                       T* out0, T* out1) {
  const int NS = nq > 32 ? 4 : 8;
  const int per = blockDim.x / NS;  // rows at a time
  const int s = threadIdx.x % NS;
  const int rot = (int)(blockIdx.x % (unsigned)nq);
  const bool vec = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  for (int q0 = 0; q0 < nq; q0 += per) {
    int q = q0 + threadIdx.x / NS;
    const bool live = q < nq;
    if (live) q = q + rot >= nq ? q + rot - nq : q + rot;
    T a0 = T(0), a1 = T(0);
    if (live) {
      const T* y = Y + (int64_t)q * n;
      if (vec) {
        const int nv = n >> 2;
#pragma unroll 8
        for (int v = s; v < nv; v += NS) {
          T yv[4], xv[4];
          // Generic loads: Y may be a shared-memory copy of the core.
          ld4(y + 4 * v, yv);
          ld4(x0 + 4 * v, xv);
#pragma unroll
          for (int i = 0; i < 4; ++i) a0 = fma(xv[i], yv[i], a0);
          if (x1) {
            ld4(x1 + 4 * v, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i) a1 = fma(xv[i], yv[i], a1);
          }
        }
      } else {
        for (int e = s; e < n; e += NS) {
          const T yy = y[e];
          a0 = fma(x0[e], yy, a0);
          if (x1) a1 = fma(x1[e], yy, a1);
        }
      }
    }
    // The NS threads of a row are consecutive lanes of one warp.
    for (int o = NS / 2; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (live && s == 0) {
      out0[q] = a0;
      if (x1) out1[q] = a1;
    }
  }
}

template <typename T>
__device__ __forceinline__ void rows_dot(const T* x, const T* Y, int n, int nq, T* out) {
  rows_dot2<T>(x, nullptr, Y, n, nq, out, nullptr);
}

// Largest core copy kept in shared memory by the kernels that dot against G.
constexpr size_t kCoreSmemBytes = 48 * 1024;
template <typename T>
__host__ __device__ inline bool core_in_smem(int64_t n) {
  return (size_t)n * sizeof(T) <= kCoreSmemBytes;
}

// The part of a multi-row update after Y: Y_r of the R <= 2 rows of the
// block (r0 .. r0 + rn - 1) is in ys (R x mu mc, Y_r[u, c] at u mc + c; rows
// past rn zero), H in hs and the old rows in fo (unless num_only). Stores Y
// (Yout), forms the numerators of the R rows with each core row read once for
// the block, then stores them (num_only) or takes the MU step.
template <typename T>
__device__ __forceinline__ void upd_rows_tail(const UpdArgs<T>& a, const T* ys, const T* hs,
                                              const T* fo, T* nm, int64_t r0, int rn, int R) {
  const int UC = a.mu * a.mc, MV = a.mv;
  if (a.Yout)
    for (int e = threadIdx.x; e < rn * UC; e += blockDim.x) a.Yout[r0 * UC + e] = ys[e];
  rows_dot2<T>(ys, R > 1 ? ys + UC : nullptr, a.Gn, UC, MV, nm, nm + MV);
  __syncthreads();
  if (a.num_only) {
    for (int e = threadIdx.x; e < rn * MV; e += blockDim.x) a.num[r0 * MV + e] = nm[e];
    return;
  }
  for (int e = threadIdx.x; e < rn * MV; e += blockDim.x) {
    const int i = e / MV, v = e % MV;
    T den = T(0);
    for (int w = 0; w < MV; ++w) den = fma(fo[i * MV + w], hs[w * MV + v], den);
    const T nv = mu_step(fo[e], nm[e], den, (T)a.eps);
    a.F[(r0 + i) * MV + v] = nv;
    write_operand(a, r0 + i, v, nv);
  }
  if (a.gate_out && r0 == 0 && threadIdx.x == 0) *a.gate_out = 1;
}

// ---------------------------------------------------------------------------
// updm: a factor update (launch_upd12) for R rows per block, the GEMMs staged by a
// three-deep cp.async ring shared by the R rows. One operand of the GEMM (the
// factor Fc) is the same for every row: it is staged once per chunk for all R
// rows. Each thread owns a TW x TW register tile of one row's Y_r (8 x 8 in
// FP32: 64 FMAs per four 16-byte shared loads, so the FMA pipe rather than
// the issue of loads and addresses bounds the GEMM); the contraction is split
// over thread groups (a warp each in the common case) whose partial tiles are
// added in group order. Then every warp forms the numerators of its core rows
// for all R rows at once (each core row read once per block, many loads in
// flight per thread, rows_dot2), and the MU step follows (or, num_only, the
// numerators are stored).
// ---------------------------------------------------------------------------
constexpr int kUpdmStages = 3;
constexpr int kUpdmRingBytes = 96 * 1024;

template <typename T>
struct Updm {
  static constexpr int TW = sizeof(T) == 4 ? 8 : 4;  // register tile edge
  static __host__ __device__ int pad(int m) { return (m + TW - 1) / TW * TW; }
  static __host__ __device__ int tiles_row(int mu, int mc) { return (pad(mu) / TW) * (pad(mc) / TW); }
  static __host__ __device__ int rows(int mu, int mc) {
    return 2 * tiles_row(mu, mc) <= kThreads / 2 ? 2 : 1;
  }
  // Elements of one staged contraction row: the shared operand once, the
  // per-row operand R times (the c side, B = P_r, unless p_first, when it is
  // the u side, A = P_r).
  static __host__ __device__ int row_elems(int mu, int mc, int R, int p_first) {
    return pad(mu) + pad(mc) + (R - 1) * (p_first ? pad(mu) : pad(mc));
  }
  // Contraction rows per stage: 64, or fewer (a multiple of 8) so that the
  // ring stays within kUpdmRingBytes.
  static __host__ __device__ int chunk(int mu, int mc, int R, int p_first) {
    int k = kUpdmRingBytes / (kUpdmStages * row_elems(mu, mc, R, p_first) * (int)sizeof(T));
    k = k > 64 ? 64 : k;
    k &= ~7;
    return k < 8 ? 8 : k;
  }
  static __host__ __device__ int groups(int mu, int mc, int R) {
    const int g = kThreads / (R * tiles_row(mu, mc));
    return g > 1 ? g : 1;
  }
  // Shared-memory elements: the ring (or the group partials, if larger), Y of
  // the R rows, H, and the old rows and numerators.
  static __host__ __device__ size_t stage_elems(int mu, int mc, int mv, int p_first, size_t* ring_out) {
    const int R = rows(mu, mc);
    const size_t ring = (size_t)kUpdmStages * chunk(mu, mc, R, p_first) * row_elems(mu, mc, R, p_first);
    const size_t red = (size_t)groups(mu, mc, R) * R * mu * (mc + 1);
    const size_t st = al4(ring > red ? ring : red);
    if (ring_out) *ring_out = st;
    return st + al4((size_t)R * mu * mc) + al4((size_t)mv * mv) + 2 * al4((size_t)R * mv);
  }
};

// Loads TW consecutive values (16-byte aligned) from shared memory.
template <int TW, typename T>
__device__ __forceinline__ void ldw(const T* p, T (&v)[TW]) {
#pragma unroll
  for (int i = 0; i < TW; i += 4) {
    T t[4];
    ld4(p + i, t);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[i + j] = t[j];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) updm_kernel(UpdArgs<T> a) {
  using U = Updm<T>;
  constexpr int TW = U::TW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MU_ = a.mu, MC = a.mc, MV = a.mv, UC = MU_ * MC;
  const int mup = U::pad(MU_), mcp = U::pad(MC);
  const int R = U::rows(MU_, MC);
  const int KC = U::chunk(MU_, MC, R, a.p_first);
  const int per = KC * U::row_elems(MU_, MC, R, a.p_first);
  const int tqc = mcp / TW, tiles_row = (mup / TW) * tqc, tiles = R * tiles_row;
  const int groups = U::groups(MU_, MC, R);
  size_t ring = 0;
  U::stage_elems(MU_, MC, MV, a.p_first, &ring);
  T* stage = sm;
  T* ys = stage + ring;                         // R x UC
  T* hs = ys + al4((size_t)R * UC);
  T* fo = hs + al4(MV * MV);                    // R x MV old rows
  T* nm = fo + al4((size_t)R * MV);             // R x MV numerators
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rn = (int)min((int64_t)R, a.nrows - r0);
  // A programmatic successor (the next sweep's first pass over X) may start
  // its prologue and its reads of X now; it waits for this grid before it
  // reads anything this kernel writes.
  pdl_trigger();

  // The row operand is P (rows of P_r) and the shared one Fc; in the chunk
  // buffers the u-side operand (A) comes first, then the c-side one (B).
  const bool a_shared = !a.p_first;  // Y = Fc^T P_r: A = Fc shared, B = P_r per row
  const int64_t lda = a_shared ? MU_ : a.pstride, ldb = a_shared ? a.pstride : MC;
  const bool vecP = aligned16(a.P, a.pstride, sizeof(T)) && ((a.prow * sizeof(T)) & 15) == 0;
  const bool vecF = aligned16(a.Fc, a_shared ? MU_ : MC, sizeof(T));
  const int na = a_shared ? 1 : R, nb = a_shared ? R : 1;
  const int nch = (a.len + KC - 1) / KC;
  // 16-byte staging: this thread's first vector (row, column) of a chunk and
  // its stride, formed once (the divisions would otherwise be redone for
  // every chunk and operand).
  constexpr int W = 16 / (int)sizeof(T);
  const int vpa = mup / W, vpb = mcp / W;
  const int ra0 = threadIdx.x / vpa, ca0 = (threadIdx.x % vpa) * W;
  const int dra = blockDim.x / vpa, dca = (blockDim.x % vpa) * W;
  const int rb0 = threadIdx.x / vpb, cb0 = (threadIdx.x % vpb) * W;
  const int drb = blockDim.x / vpb, dcb = (blockDim.x % vpb) * W;
  // Offsets within a chunk in 32 bits (used when KC row strides fit).
  auto stage_fast = [&](T* dst, int lds, const T* src, int64_t ldg, int tn, int vrows, int vcols,
                        int r, int cc, int dr, int dc) {
    const int nv = tn * (lds / W);
    const int ldg32 = (int)ldg;
    int so = r * ldg32 + cc, doff = r * lds + cc;
    const int dso = dr * ldg32 + dc, ddo = dr * lds + dc;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      int valid = r < vrows ? vcols - cc : 0;
      valid = valid < 0 ? 0 : (valid > W ? W : valid);
      cp_vec(dst + doff, valid ? src + so : src, valid);
      r += dr;
      cc += dc;
      so += dso;
      doff += ddo;
      if (cc >= lds) {
        cc -= lds;
        ++r;
        so += ldg32 - lds;  // (the shared offset needs no correction: its rows are lds long)
      }
    }
  };
  auto issue = [&](int c) {
    T* st = stage + (c % kUpdmStages) * per;
    const int t0 = c * KC, tn = min(KC, a.len - t0);
    for (int i = 0; i < na; ++i) {
      const T* src = a_shared ? a.Fc : a.P + (r0 + (i < rn ? i : 0)) * a.prow;
      const bool vec = a_shared ? vecF : vecP;
      const int vr = i < rn || a_shared ? tn : 0;
      if (vec && (mup % W) == 0 && lda * KC < (1LL << 31))
        stage_fast(st + i * KC * mup, mup, src + (int64_t)t0 * lda, lda, tn, vr, MU_, ra0, ca0,
                   dra, dca);
      else
        stage_tile(st + i * KC * mup, mup, src + (int64_t)t0 * lda, lda, tn, mup, vr, MU_, vec);
    }
    T* sb = st + na * KC * mup;
    for (int i = 0; i < nb; ++i) {
      const T* src = a_shared ? a.P + (r0 + (i < rn ? i : 0)) * a.prow : a.Fc;
      const bool vec = a_shared ? vecP : vecF;
      const int vr = i < rn || !a_shared ? tn : 0;
      if (vec && (mcp % W) == 0 && ldb * KC < (1LL << 31))
        stage_fast(sb + i * KC * mcp, mcp, src + (int64_t)t0 * ldb, ldb, tn, vr, MC, rb0, cb0,
                   drb, dcb);
      else
        stage_tile(sb + i * KC * mcp, mcp, src + (int64_t)t0 * ldb, ldb, tn, mcp, vr, MC, vec);
    }
    cp_commit();
  };
  // Everything but the GEMM operands is requested first; the first wait
  // covers it.
  if (!a.num_only) {
    cp_flat(hs, a.H, MV * MV);
    cp_flat(fo, a.F + r0 * MV, (int64_t)rn * MV);
  }
  cp_commit();
  for (int c = 0; c < kUpdmStages - 1; ++c) {
    if (c < nch) issue(c);
    else cp_commit();  // empty groups keep the wait count uniform
  }
  const int g = threadIdx.x / tiles, tl = threadIdx.x % tiles;
  const bool act = g < groups;
  const int ri = tl / tiles_row, tt = tl % tiles_row;
  const int u0 = (tt / tqc) * TW, c0 = (tt % tqc) * TW;
  T acc[TW][TW];
#pragma unroll
  for (int i = 0; i < TW; ++i)
#pragma unroll
    for (int j = 0; j < TW; ++j) acc[i][j] = T(0);
  for (int c = 0; c < nch; ++c) {
    if (c + kUpdmStages - 1 < nch) issue(c + kUpdmStages - 1);
    else cp_commit();
    cp_wait<kUpdmStages - 1>();
    __syncthreads();
    if (act) {
      const T* st = stage + (c % kUpdmStages) * per;
      const T* A = st + (a_shared ? 0 : ri * KC * mup) + u0;
      const T* B = st + na * KC * mup + (a_shared ? ri * KC * mcp : 0) + c0;
      const int kn = min(KC, a.len - c * KC);
      // One k at a time: TW x TW independent accumulators already hide the
      // FMA latency, and the registers stay free for them.
#pragma unroll 1
      for (int k = g; k < kn; k += groups) {
        T x[TW], y[TW];
        ldw<TW>(A + k * mup, x);
        ldw<TW>(B + k * mcp, y);
#pragma unroll
        for (int i = 0; i < TW; ++i)
#pragma unroll
          for (int j = 0; j < TW; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  cp_wait<0>();
  __syncthreads();
  // The group partials, rows padded to MC + 1 so that the threads of a warp
  // (tiles TW rows apart) store to different banks.
  T* red = stage;  // the ring is free after the last barrier
  const int ldr = MC + 1, plane = MU_ * ldr;
  if (act) {
#pragma unroll
    for (int i = 0; i < TW; ++i)
#pragma unroll
      for (int j = 0; j < TW; ++j)
        if (u0 + i < MU_ && c0 + j < MC)
          red[((size_t)g * R + ri) * plane + (u0 + i) * ldr + c0 + j] = acc[i][j];
  }
  __syncthreads();
  {
    // e = (i, u, cc) walked by increments (no division per entry).
    int i = threadIdx.x / UC, u = (threadIdx.x % UC) / MC, cc = threadIdx.x % MC;
    const int di = blockDim.x / UC, du = (blockDim.x % UC) / MC, dc = blockDim.x % MC;
    for (int e = threadIdx.x; e < R * UC; e += blockDim.x) {
      T v = T(0);
      for (int q = 0; q < groups; ++q) v += red[((size_t)q * R + i) * plane + u * ldr + cc];
      ys[e] = v;
      i += di;
      u += du;
      cc += dc;
      if (cc >= MC) {
        cc -= MC;
        ++u;
      }
      if (u >= MU_) {
        u -= MU_;
        ++i;
      }
    }
  }
  __syncthreads();
  upd_rows_tail<T>(a, ys, hs, fo, nm, r0, rn, R);
}

// ---------------------------------------------------------------------------
// updt: the update of updm with the GEMMs on the tensor cores, for FP32 data
// with mu, mc <= 32. A block takes two rows; warp w works on row w / 4 and on
// every fourth 8-deep step of the contraction, holding the whole zero-padded
// 32 x 32 tile Z_r = Fc^T P_r (Y_r, or Y_r^T when p_first) in registers. A
// step is eight mma.sync m16n8k8 (TF32 operands, FP32 accumulation), or 24
// with SPLIT = 3, which splits every operand x into x_hi = tf32(x) and x_lo =
// tf32(x - x_hi) and accumulates x_lo y_hi + x_hi y_lo + x_hi y_hi (the
// dropped x_lo y_lo is below FP32 rounding). The four partial tiles of a row
// are added in warp order, so results are deterministic. One thread stages
// the operands with the TMA unit, 64 contraction rows of Fc and of both rows'
// P_r per stage, four stages deep (the tensor maps zero-fill every edge).
// Y_r goes to UpdArgs::ybuf, where numu_kernel takes it. The fragments and
// the layout of a tile in registers are mma32.cuh's.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 2;                               // rows per block
constexpr int kTcWarpsPerRow = kThreads / 32 / kTcRows;  // contraction split
constexpr int kTcKC = 64;                                // contraction rows per stage
constexpr int kTcStages = 4;
constexpr int kTcBox = kTcKC * 32;                       // one operand's box (floats)
constexpr int kTcStage = (1 + kTcRows) * kTcBox;         // Fc's box, then the rows'
constexpr uint32_t kTcStageBytes = kTcStage * 4;
constexpr int kTcZ = 32 * 32;                            // one partial tile (mma32::tile_index)

__host__ __device__ inline size_t updt_ring_floats() {
  const size_t ring = (size_t)kTcStages * kTcStage;
  const size_t red = (size_t)kTcRows * kTcWarpsPerRow * kTcZ;
  return al4(ring > red ? ring : red);
}
// Floats of dynamic shared memory, with 1024 bytes of slack to align the ring.
__host__ __device__ inline size_t updt_smem_floats(int mu, int mc) {
  return 256 + updt_ring_floats() + al4((size_t)kTcRows * mu * mc);
}

template <int SPLIT>
__global__ void __launch_bounds__(kThreads, 2)
    updt_kernel(UpdArgs<float> a, const __grid_constant__ CUtensorMap map_f,
                const __grid_constant__ CUtensorMap map_p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kTcStages];
  constexpr int R = kTcRows;
  const int MU_ = a.mu, MC = a.mc, UC = MU_ * MC;
  // The ring starts on a 1024-byte boundary (the swizzle's period).
  const uint32_t pad = (1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u;
  float* stage = reinterpret_cast<float*>(smem_raw + pad);
  float* ys = stage + updt_ring_floats();       // R x UC
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rn = (int)min((int64_t)R, a.nrows - r0);
  pdl_trigger();  // as in updm

  // Stage c holds contraction rows c KC .. c KC + KC - 1 of Fc (box 32 x KC)
  // and of the block's two row operands (box 32 x KC x 2); the TMA unit reads
  // entries outside Fc, P or the contraction as zero.
  const int nch = (a.len + kTcKC - 1) / kTcKC;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kTcStages; ++k) tma::mbar_init(&full[k], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int c) {  // one thread
    float* st = stage + (c % kTcStages) * kTcStage;
    uint64_t* bar = &full[c % kTcStages];
    tma::mbar_expect_tx(bar, kTcStageBytes);
    tma::load_2d(st, &map_f, 0, c * kTcKC, bar);
    tma::load_3d(st + kTcBox, &map_p, 0, c * kTcKC, (int)r0, bar);
  };
  if (threadIdx.x == 0)
    for (int c = 0; c < kTcStages - 1 && c < nch; ++c) issue(c);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ri = warp / kTcWarpsPerRow, wk = warp % kTcWarpsPerRow;
  const int off0 = mma32::frag_off(lane, 0), off1 = mma32::frag_off(lane, 1);
  float acc[2][4][4];
  mma32::zero(acc);
  for (int c = 0; c < nch; ++c) {
    // The slot of stage c + 2 was released by the barrier ending step c - 1.
    if (threadIdx.x == 0 && c + kTcStages - 1 < nch) issue(c + kTcStages - 1);
    bool ok = tma::mbar_wait(&full[c % kTcStages], (c / kTcStages) & 1, a.err);
    if (ok) {
      const float* sa = stage + (c % kTcStages) * kTcStage;
      const float* sb = sa + (1 + ri) * kTcBox;
      const int kn8 = (min(kTcKC, a.len - c * kTcKC) + 7) / 8;
#pragma unroll 2
      for (int ks = wk; ks < kn8; ks += kTcWarpsPerRow)
        mma32::step<SPLIT>(acc, sa + ks * 256, sb + ks * 256, off0, off1);
    }
    if (!__syncthreads_and(ok)) {
      // A copy did not arrive (the flag is raised): wait, bounded, for the
      // stages still in flight so that none lands after the block has exited.
      if (threadIdx.x == 0)
        for (int d = c; d < nch && d < c + kTcStages; ++d)
          tma::mbar_wait(&full[d % kTcStages], (d / kTcStages) & 1, nullptr);
      return;
    }
  }
  // The partial tiles, then the row's four partials added in warp order into
  // Y_r (Z_r, or Z_r^T when p_first) in ys.
  float* red = stage;  // every stage has landed and been read
  mma32::store(red + (ri * kTcWarpsPerRow + wk) * kTcZ, acc, lane);
  __syncthreads();
  for (int row = warp; row < R * MU_; row += kThreads / 32) {
    const int i = row / MU_, u = row - i * MU_;
    const float* zi = red + i * kTcWarpsPerRow * kTcZ;
    for (int cc = lane; cc < MC; cc += 32) {
      const int o = a.p_first ? mma32::tile_index(cc, u) : mma32::tile_index(u, cc);
      float v = zi[o];
#pragma unroll
      for (int w = 1; w < kTcWarpsPerRow; ++w) v += zi[o + w * kTcZ];
      ys[i * UC + u * MC + cc] = v;
    }
  }
  __syncthreads();
  // Y of the block's rows to the numerator kernel (UC % 4 == 0).
  float4* yo = reinterpret_cast<float4*>(a.ybuf + r0 * UC);
  for (int e = threadIdx.x; e < rn * UC / 4; e += kThreads)
    yo[e] = reinterpret_cast<const float4*>(ys)[e];
}

// ---------------------------------------------------------------------------
// numu: the numerators and the MU step of the tensor-core update form, eight
// rows per block. Num[r, v] = <Y_r, Gn[v]> for the block's rows is one GEMM,
// Num (8 x mv) = Y (8 x UC) Gn^T, on the tensor cores (mma.sync m16n8k8 with
// the rows as M rows 0..7 and zeros as rows 8..15): warp w of 16 takes every
// 16th 16-deep step of the contraction with all mv <= 32 columns, and the 16
// partial results are added in warp order. The core arrives in shared memory
// by one bulk copy per row (rows padded to a pitch of 4 mod 8 16-byte units,
// so the fragment loads below are free of bank conflicts) while every thread
// loads its entries of Y: from the GEMM form's buffer (ybuf) or as the sum of
// the pass's shares (added in share order, and stored to Yout when asked),
// all of a thread's loads in flight at once. Then the MU step of the rows, or
// (num_only) their numerators. SPLIT as in mma32::step.
//
// Fragments: thread (g, t) = (lane / 4, lane % 4) takes entries k0 + 4t ..
// k0 + 4t + 3 of row g of Y and of rows 8j + g of Gn (16-byte loads); MMA
// h = 0, 1 of the step takes k = t from entry 4t + 2h and k = t + 4 from
// entry 4t + 2h + 1, the same for both operands.
// ---------------------------------------------------------------------------
constexpr int kNuRows = 8;
constexpr int kNuThreads = 512;
constexpr int kNuWarps = kNuThreads / 32;
constexpr int kNuSteps = 4;  // 16-deep steps per warp at most (UC <= 1024)

// Row pitch (floats) of the core in shared memory.
__host__ __device__ inline int numu_pitch(int uc) {
  const int u = uc / 4;
  return 4 * (u + ((4 - u % 8) + 8) % 8);
}
__host__ __device__ inline size_t numu_smem_floats(int mu, int mc, int mv) {
  return (size_t)mv * numu_pitch(mu * mc) + (size_t)kNuWarps * kNuRows * 32 +
         al4((size_t)mv * mv) + 2 * al4((size_t)kNuRows * mv);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

template <int SPLIT>
__device__ __forceinline__ void numu_mma(float (&acc)[4][4], float4 y, const float4 (&gv)[4]) {
  const float ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t ah[4] = {mma32::tf32_rn(ya[2 * h]), 0u, mma32::tf32_rn(ya[2 * h + 1]), 0u};
    uint32_t al[4] = {0u, 0u, 0u, 0u};
    if constexpr (SPLIT == 3) {
      al[0] = mma32::tf32_rn(ya[2 * h] - __uint_as_float(ah[0]));
      al[2] = mma32::tf32_rn(ya[2 * h + 1] - __uint_as_float(ah[2]));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float g0 = h ? gv[j].z : gv[j].x, g1 = h ? gv[j].w : gv[j].y;
      const uint32_t bh0 = mma32::tf32_rn(g0), bh1 = mma32::tf32_rn(g1);
      if constexpr (SPLIT == 3) {
        const uint32_t bl0 = mma32::tf32_rn(g0 - __uint_as_float(bh0));
        const uint32_t bl1 = mma32::tf32_rn(g1 - __uint_as_float(bh1));
        mma32::mma_tf32(acc[j], al, bh0, bh1);
        mma32::mma_tf32(acc[j], ah, bl0, bl1);
      }
      mma32::mma_tf32(acc[j], ah, bh0, bh1);
    }
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(kNuThreads, 1) numu_kernel(UpdArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t gbar;
  const int UC = a.mu * a.mc, MV = a.mv, pitch = numu_pitch(UC);
  float* gs = reinterpret_cast<float*>(smem_raw);     // MV rows of the core, pitch apart
  float* red = gs + (size_t)MV * pitch;              // 16 warps x 8 rows x 32
  float* hs = red + kNuWarps * kNuRows * 32;
  float* fo = hs + al4((size_t)MV * MV);             // old rows
  float* nm = fo + al4((size_t)kNuRows * MV);        // numerators
  const int64_t r0 = (int64_t)blockIdx.x * kNuRows;
  const int rn = (int)min((int64_t)kNuRows, a.nrows - r0);
  pdl_trigger();  // as in updm
  if (threadIdx.x == 0) {
    tma::mbar_init(&gbar, 1);
    tma::mbar_init_fence();
  }
  __syncthreads();  // the barrier is initialised before anyone waits on it
  if (threadIdx.x == 0) {
    tma::mbar_expect_tx(&gbar, (uint32_t)(MV * UC * 4));
    for (int v = 0; v < MV; ++v)
      tma::load_bulk(gs + (size_t)v * pitch, a.Gn + (int64_t)v * UC, (uint32_t)(UC * 4), &gbar);
  }
  // Launched as a programmatic dependent: the kernel before it on the stream
  // (a pass, the GEMM form, a Gram kernel) may still run until here. None of
  // them writes the core, so its copy above overlaps their tail; everything
  // below may be theirs.
  pdl_wait();
  if (!a.num_only) {
    cp_flat(hs, a.H, MV * MV);
    cp_flat(fo, a.F + r0 * MV, (int64_t)rn * MV);
  }
  cp_commit();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int g = lane >> 2, t = lane & 3;
  const int np = a.Ypart ? a.nparts : 1;
  const bool rowok = g < rn;
  const float* yrow = (a.Ypart ? a.Ypart : a.ybuf) + (rowok ? (r0 + g) * np * UC : 0);
  float* yout = (a.Ypart && a.Yout && rowok) ? a.Yout + (r0 + g) * UC : nullptr;
  const int nsteps = (UC + 15) / 16;
  // This thread's entries of Y for its steps, all loads in flight together.
  float4 y[kNuSteps];
  bool live[kNuSteps];
#pragma unroll
  for (int q = 0; q < kNuSteps; ++q) {
    const int k = (warp + q * kNuWarps) * 16 + 4 * t;
    live[q] = warp + q * kNuWarps < nsteps && k < UC && rowok;  // UC % 4 == 0
    y[q] = live[q] ? *reinterpret_cast<const float4*>(yrow + k) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int h0 = 1; h0 < np; h0 += 4) {
    float4 z[kNuSteps][4];
#pragma unroll
    for (int q = 0; q < kNuSteps; ++q) {
      const int k = (warp + q * kNuWarps) * 16 + 4 * t;
#pragma unroll
      for (int p = 0; p < 4; ++p)
        z[q][p] = live[q] && h0 + p < np
                      ? *reinterpret_cast<const float4*>(yrow + (int64_t)(h0 + p) * UC + k)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kNuSteps; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p)
        if (h0 + p < np) y[q] = add4(y[q], z[q][p]);
  }
  if (yout) {
#pragma unroll
    for (int q = 0; q < kNuSteps; ++q)
      if (live[q]) *reinterpret_cast<float4*>(yout + (warp + q * kNuWarps) * 16 + 4 * t) = y[q];
  }
  const bool ok = tma::mbar_wait(&gbar, 0, a.err);
  if (!__syncthreads_and(ok)) {
    // The core did not arrive (the flag is raised): wait, bounded, for the
    // copies still in flight so that none lands after the block has exited.
    if (threadIdx.x == 0) tma::mbar_wait(&gbar, 0, nullptr);
    cp_wait<0>();
    return;
  }
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
  for (int q = 0; q < kNuSteps; ++q) {
    const int st = warp + q * kNuWarps;
    if (st >= nsteps) break;
    const int k = st * 16 + 4 * t;
    float4 gv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = 8 * j + g;
      gv[j] = (k < UC && n < MV) ? *reinterpret_cast<const float4*>(gs + n * pitch + k)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    numu_mma<SPLIT>(acc, y[q], gv);
  }
  // Partial numerators of the warp: rows g (c0, c1; rows 8..15 are padding).
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    red[(warp * kNuRows + g) * 32 + 8 * j + 2 * t] = acc[j][0];
    red[(warp * kNuRows + g) * 32 + 8 * j + 2 * t + 1] = acc[j][1];
  }
  cp_wait<0>();
  __syncthreads();
  for (int e = threadIdx.x; e < rn * MV; e += kNuThreads) {
    const int r = e / MV, v = e - r * MV;
    float n = red[r * 32 + v];
#pragma unroll
    for (int w = 1; w < kNuWarps; ++w) n += red[(w * kNuRows + r) * 32 + v];
    nm[e] = n;
  }
  __syncthreads();
  if (a.num_only) {
    for (int e = threadIdx.x; e < rn * MV; e += kNuThreads) a.num[r0 * MV + e] = nm[e];
    return;
  }
  for (int e = threadIdx.x; e < rn * MV; e += kNuThreads) {
    const int i = e / MV, v = e - i * MV;
    float den = 0.f;
    for (int w = 0; w < MV; ++w) den = fmaf(fo[i * MV + w], hs[w * MV + v], den);
    const float nv = mu_step(fo[e], nm[e], den, (float)a.eps);
    a.F[(r0 + i) * MV + v] = nv;
    write_operand(a, r0 + i, v, nv);
  }
  if (a.gate_out && r0 == 0 && threadIdx.x == 0) *a.gate_out = 1;
}

// ---------------------------------------------------------------------------
// upds: a factor update from the pass's shares of Y_r, two rows per block
// (each core row read once for both, as in updm): Y_r = the sum of its
// nparts shares in order h = 0 .. nparts - 1, then upd_rows_tail.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) upds_kernel(UpdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int R = 2;
  const int UC = a.mu * a.mc, MV = a.mv;
  T* ys = sm;                                  // R x UC
  T* hs = ys + al4((size_t)R * UC);
  T* fo = hs + al4((size_t)MV * MV);           // R x MV old rows
  T* nm = fo + al4((size_t)R * MV);            // R x MV numerators
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rn = (int)min((int64_t)R, a.nrows - r0);
  pdl_trigger();  // as in updm
  if (!a.num_only) {
    cp_flat(hs, a.H, MV * MV);
    cp_flat(fo, a.F + r0 * MV, (int64_t)rn * MV);
  }
  cp_commit();
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if ((UC & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Ypart) & 15) == 0) {
      // 16-byte vectors, two per thread at a time, with the loads of four
      // shares of both in flight before they are added (in share order).
      const int nv = R * UC / 4;
      for (int v0 = threadIdx.x; v0 < nv; v0 += 2 * blockDim.x) {
        float4 y[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
        for (int h0 = 0; h0 < a.nparts; h0 += 4) {
          float4 t[2][4];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int v = v0 + k * blockDim.x, i = 4 * v / UC;
            const float* yp = a.Ypart + ((r0 + i) * a.nparts + h0) * UC + (4 * v - i * UC);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              t[k][q] = (v < nv && i < rn && h0 + q < a.nparts)
                            ? *reinterpret_cast<const float4*>(yp + (int64_t)q * UC)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (h0 + q == 0) {
                y[k] = t[k][q];
              } else if (h0 + q < a.nparts) {
                y[k].x += t[k][q].x; y[k].y += t[k][q].y;
                y[k].z += t[k][q].z; y[k].w += t[k][q].w;
              }
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (v0 + k * blockDim.x < nv)
            *reinterpret_cast<float4*>(ys + 4 * (v0 + k * blockDim.x)) = y[k];
      }
      done = true;
    }
  }
  if (!done) {
    for (int e = threadIdx.x; e < R * UC; e += blockDim.x) {
      const int i = e / UC, f = e - i * UC;
      T y = T(0);
      if (i < rn) {
        const T* yp = a.Ypart + (r0 + i) * a.nparts * UC + f;
        y = yp[0];
        for (int h = 1; h < a.nparts; ++h) y += yp[(int64_t)h * UC];
      }
      ys[e] = y;
    }
  }
  cp_wait<0>();
  __syncthreads();
  upd_rows_tail<T>(a, ys, hs, fo, nm, r0, rn, R);
}

// ---------------------------------------------------------------------------
// mu_rows: the MU step of a split update, kThreads / mv rows per block.
//   F[r, v] <- MU(F[r, v], num[r, v], sum_w F[r, w] H[w, v])
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) mu_rows_kernel(UpdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MV = a.mv, R = kThreads / MV;
  pdl_trigger();  // as in updm
  T* hs = sm;                  // MV x MV
  T* fo = hs + al4(MV * MV);   // R x MV: the old rows
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rn = (int)min((int64_t)R, a.nrows - r0);
  cp_flat(hs, a.H, MV * MV);
  cp_flat(fo, a.F + r0 * MV, (int64_t)rn * MV);
  cp_commit();
  cp_wait<0>();
  __syncthreads();
  const int t = threadIdx.x;
  if (t < rn * MV) {
    const int rr = t / MV, v = t % MV;
    T den = T(0);
    for (int w = 0; w < MV; ++w) den = fma(fo[rr * MV + w], hs[w * MV + v], den);
    const T nv = mu_step(fo[t], a.num[r0 * MV + t], den, (T)a.eps);
    a.F[r0 * MV + t] = nv;
    write_operand(a, r0 + rr, v, nv);
  }
  if (a.gate_out && r0 == 0 && t == 0) *a.gate_out = 1;
}

// ---------------------------------------------------------------------------
// hmat: H_n for one mode (and optionally the W slices), one block per p.
//   W[p] = S_u G[p] S_v;  H[p, q] = <W[p], G[q]>
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) hmat_kernel(HArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int U = a.mu, V = a.mv, P = a.mp, UV = U * V;
  const bool gsm = core_in_smem<T>((int64_t)P * UV);
  const size_t st_u = a.fu ? gemm_stage_elems(U, U, (int)sizeof(T), (int)a.nu) : 0;
  const size_t st_v = a.fv ? gemm_stage_elems(V, V, (int)sizeof(T), (int)a.nv) : 0;
  T* stage = sm;
  T* su = stage + (st_u > st_v ? st_u : st_v);
  T* sv = su + al4(U * U);
  T* gp = sv + al4(V * V);
  T* tp = gp + al4(UV);
  T* wp = tp + al4(UV);
  T* gs = wp + al4(UV);  // P x U x V when it fits
  const int p = blockIdx.x;

  if (!a.fu) cp_flat(su, a.su, U * U);
  if (!a.fv) cp_flat(sv, a.sv, V * V);
  if (gsm) cp_flat(gs, a.Gn, (int64_t)P * UV);
  else cp_flat(gp, a.Gn + (int64_t)p * UV, UV);
  cp_commit();
  if (a.fu)
    gemm_tn_block(a.fu, U, U, a.fu, U, U, (int)a.nu, gemm_kch(U, U, (int)sizeof(T), (int)a.nu),
                  su, stage);
  if (a.fv)
    gemm_tn_block(a.fv, V, V, a.fv, V, V, (int)a.nv, gemm_kch(V, V, (int)sizeof(T), (int)a.nv),
                  sv, stage);
  if (!a.fu && !a.fv) {
    cp_wait<0>();
    __syncthreads();
  }
  const T* g = gsm ? gs + (int64_t)p * UV : gp;
  if (p == 0 && a.su_out && a.fu)
    for (int e = threadIdx.x; e < U * U; e += blockDim.x) a.su_out[e] = su[e];
  if (p == 0 && a.sv_out && a.fv)
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) a.sv_out[e] = sv[e];
  smem_gemm(su, g, tp, U, U, V);  // S_u G[p]
  __syncthreads();
  smem_gemm(tp, sv, wp, U, V, V);  // (S_u G[p]) S_v
  __syncthreads();
  if (a.Wout)
    for (int e = threadIdx.x; e < UV; e += blockDim.x)
      a.Wout[(int64_t)p * a.w_sp + (int64_t)(e / V) * a.w_su + (int64_t)(e % V) * a.w_sv] = wp[e];
  rows_dot(wp, gsm ? (const T*)gs : a.Gn, UV, P, a.H + (int64_t)p * P);
}

// ---------------------------------------------------------------------------
// core_a: one block per mode-1 index a (no block depends on another):
//   S3 = F3^T F3;  M[a] = Y3[:, a, :]^T F3 (= (X x_1 F1^T x_2 F2^T x_3 F3^T)[a]);
//   D[a] = W3[a] x_3 S3;  G[a] <- MU(G[a], M[a], D[a]);  W1[a] = S2 G[a] S3
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) core_a_kernel(CoreArgs<T> a) {
  if (a.gate && *a.gate == 0) return;  // no sweep since the last core update
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int m1 = a.m1, m2 = a.m2, m3 = a.m3;
  const int bc = m2 * m3;
  const size_t st3 = gemm_stage_elems(m3, m3, (int)sizeof(T), (int)a.n3);
  const size_t stm = gemm_stage_elems(m2, m3, (int)sizeof(T), (int)a.n3);
  T* stage = sm;
  T* s2 = stage + (st3 > stm ? st3 : stm);  // m2 x m2
  T* s3 = s2 + al4(m2 * m2);                  // m3 x m3
  T* ma = s3 + al4(m3 * m3);                  // bc: M[a]
  T* wa = ma + al4(bc);                       // bc: W3[a], then scratch
  T* ga = wa + al4(bc);                       // bc: G[a]
  const int aa = blockIdx.x;
  const int64_t off = (int64_t)aa * bc;

  cp_flat(s2, a.S2, m2 * m2);
  cp_flat(wa, a.W3 + off, bc);
  cp_flat(ga, a.G + off, bc);
  cp_commit();
  gemm_tn_block(a.F3, m3, m3, a.F3, m3, m3, (int)a.n3,
                gemm_kch(m3, m3, (int)sizeof(T), (int)a.n3), s3, stage);
  gemm_tn_block(a.Y3 + (int64_t)aa * m2, (int64_t)m1 * m2, m2, a.F3, m3, m3, (int)a.n3,
                gemm_kch(m2, m3, (int)sizeof(T), (int)a.n3), ma, stage);
  if (aa == 0)
    for (int e = threadIdx.x; e < m3 * m3; e += blockDim.x) a.S3_out[e] = s3[e];
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {
    const int b = e / m3, c = e % m3;
    T d = T(0);
    for (int w = 0; w < m3; ++w) d = fma(wa[b * m3 + w], s3[w * m3 + c], d);
    const T gv = mu_step(ga[e], ma[e], d, (T)a.eps);
    ga[e] = gv;
    a.G[off + e] = gv;
    a.G2[((int64_t)b * m1 + aa) * m3 + c] = gv;  // G permuted to (m2, m1, m3)
    a.G3[((int64_t)c * m1 + aa) * m2 + b] = gv;  // G permuted to (m3, m1, m2)
    a.Mout[off + e] = ma[e];
  }
  __syncthreads();
  smem_gemm(s2, ga, wa, m2, m2, m3);  // S2 G[a]
  __syncthreads();
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {  // W1[a] = (S2 G[a]) S3
    const int b = e / m3, c = e % m3;
    T v = T(0);
    for (int w = 0; w < m3; ++w) v = fma(wa[b * m3 + w], s3[w * m3 + c], v);
    a.W1[off + e] = v;
  }
}

// ---------------------------------------------------------------------------
// Block GEMMs on the tensor cores for the kernels beside the passes (hmat,
// core_a): Z_p = A_p^T B for p < NP (32 x 32, zero past the operands' width),
// summed over `len` contraction rows. B and every A_p are row sets of at most
// 32 FP32 entries that the TMA unit reads (box of 32 entries x 64 rows at
// (0, t0) of a 2-D map, or (0, t0, row) of a 3-D one) into a three-deep ring,
// one stage per 64 rows; an A_p without a map is B itself (a Gram). The eight
// warps split over the products and over every (8 / NP)-th 8-deep step of the
// contraction (mma32::step, SPLIT as there) and their partial tiles are added
// in warp order into out[p] (entry (s, c) at s ld + c, for s < ms[p], c < mc).
// Called once per block, by every thread; false (with *err raised) when a
// copy did not arrive, after waiting (bounded) for the stages in flight.
// ---------------------------------------------------------------------------
struct TcOperand {
  const CUtensorMap* map;  // NULL: the B operand itself
  int row;                 // third coordinate of a 3-D map, -1 for a 2-D map
};

constexpr int kTbBox = 64 * 32;  // floats in one operand box
constexpr int kTbStages = 3;

// Ring floats for NP products (also room for the partial tiles).
__host__ __device__ inline size_t tc_block_ring_floats(int np) {
  const size_t ring = (size_t)kTbStages * (1 + np) * kTbBox, red = (size_t)8 * 1024;
  return ring > red ? ring : red;
}

__device__ __forceinline__ void tma_box(float* dst, const TcOperand& o, int t0, uint64_t* bar) {
  if (o.row < 0) tma::load_2d(dst, o.map, 0, t0, bar);
  else tma::load_3d(dst, o.map, 0, t0, o.row, bar);
}

template <int SPLIT, int NP>
__device__ bool tc_block_gemm(const TcOperand (&A)[NP], const TcOperand& B, int len,
                              float* ring, uint64_t* bars, float* const (&out)[NP], int ld,
                              const int (&ms)[NP], int mc, int* err) {
  constexpr int WPP = 8 / NP;  // warps per product
  int nbox = 1;
#pragma unroll
  for (int p = 0; p < NP; ++p) nbox += A[p].map ? 1 : 0;
  const int per = (1 + NP) * kTbBox;
  const uint32_t bytes = (uint32_t)nbox * kTbBox * 4;
  const int nch = (len + 63) / 64;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kTbStages; ++k) tma::mbar_init(&bars[k], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int c) {  // one thread
    float* st = ring + (c % kTbStages) * per;
    uint64_t* bar = &bars[c % kTbStages];
    tma::mbar_expect_tx(bar, bytes);
    tma_box(st, B, c * 64, bar);
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (A[p].map) tma_box(st + (1 + p) * kTbBox, A[p], c * 64, bar);
  };
  if (threadIdx.x == 0)
    for (int c = 0; c < kTbStages - 1 && c < nch; ++c) issue(c);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int p = warp / WPP, wk = warp % WPP;
  const int off0 = mma32::frag_off(lane, 0), off1 = mma32::frag_off(lane, 1);
  float acc[2][4][4];
  mma32::zero(acc);
  bool aself = true;
#pragma unroll
  for (int q = 0; q < NP; ++q)
    if (q == p) aself = A[q].map == nullptr;
  for (int c = 0; c < nch; ++c) {
    if (threadIdx.x == 0 && c + kTbStages - 1 < nch) issue(c + kTbStages - 1);
    const bool ok = tma::mbar_wait(&bars[c % kTbStages], (c / kTbStages) & 1, err);
    if (ok) {
      const float* sb = ring + (c % kTbStages) * per;
      const float* sa = aself ? sb : sb + (1 + p) * kTbBox;
      const int kn8 = (min(64, len - c * 64) + 7) / 8;
      for (int ks = wk; ks < kn8; ks += WPP)
        mma32::step<SPLIT>(acc, sa + ks * 256, sb + ks * 256, off0, off1);
    }
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0)
        for (int d = c; d < nch && d < c + kTbStages; ++d)
          tma::mbar_wait(&bars[d % kTbStages], (d / kTbStages) & 1, nullptr);
      return false;
    }
  }
  float* red = ring;  // every stage has landed and been read
  mma32::store(red + warp * 1024, acc, lane);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    for (int e = threadIdx.x; e < ms[q] * mc; e += blockDim.x) {
      const int s = e / mc, cc = e - s * mc, o = mma32::tile_index(s, cc);
      const float* z = red + q * WPP * 1024 + o;
      float v = z[0];
#pragma unroll
      for (int w = 1; w < WPP; ++w) v += z[w * 1024];
      out[q][s * ld + cc] = v;
    }
  }
  __syncthreads();
  return true;
}

// hmat on the tensor cores: the Gram of the factor given (fu or fv) by
// tc_block_gemm, the rest as in hmat_kernel. FP32, U, V, P <= 32.
template <int SPLIT>
__global__ void __launch_bounds__(kThreads)
    hmat_tc_kernel(HArgs<float> a, const __grid_constant__ CUtensorMap map_f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kTbStages];
  const uint32_t pad = (1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u;
  float* ring = reinterpret_cast<float*>(smem_raw + pad);
  const int U = a.mu, V = a.mv, P = a.mp, UV = U * V;
  float* su = ring + tc_block_ring_floats(1);
  float* sv = su + al4(U * U);
  float* gp = sv + al4(V * V);
  float* tp = gp + al4(UV);
  float* wp = tp + al4(UV);
  const int p = blockIdx.x;
  if (!a.fu) cp_flat(su, a.su, U * U);
  if (!a.fv) cp_flat(sv, a.sv, V * V);
  cp_flat(gp, a.Gn + (int64_t)p * UV, UV);
  cp_commit();
  const TcOperand self[1] = {{nullptr, -1}};
  const TcOperand fb{&map_f, -1};
  float* const outs[1] = {a.fu ? su : sv};
  const int mss[1] = {a.fu ? U : V};
  const bool ok = tc_block_gemm<SPLIT, 1>(self, fb, (int)(a.fu ? a.nu : a.nv), ring, bars, outs,
                                          a.fu ? U : V, mss, a.fu ? U : V, a.err);
  cp_wait<0>();
  __syncthreads();
  if (!ok) return;
  if (p == 0 && a.su_out && a.fu)
    for (int e = threadIdx.x; e < U * U; e += blockDim.x) a.su_out[e] = su[e];
  if (p == 0 && a.sv_out && a.fv)
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) a.sv_out[e] = sv[e];
  smem_gemm(su, gp, tp, U, U, V);  // S_u G[p]
  __syncthreads();
  smem_gemm(tp, sv, wp, U, V, V);  // (S_u G[p]) S_v
  __syncthreads();
  if (a.Wout)
    for (int e = threadIdx.x; e < UV; e += blockDim.x)
      a.Wout[(int64_t)p * a.w_sp + (int64_t)(e / V) * a.w_su + (int64_t)(e % V) * a.w_sv] = wp[e];
  rows_dot(wp, a.Gn, UV, P, a.H + (int64_t)p * P);
}

// core_a on the tensor cores: S3 = F3^T F3 and M[a] = Y3[:, a, :]^T F3 in one
// tc_block_gemm (both products share F3's boxes), the rest as in core_a_kernel.
template <int SPLIT>
__global__ void __launch_bounds__(kThreads)
    core_a_tc_kernel(CoreArgs<float> a, const __grid_constant__ CUtensorMap map_f3,
                     const __grid_constant__ CUtensorMap map_y3) {
  if (a.gate && *a.gate == 0) return;  // no sweep since the last core update
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kTbStages];
  const uint32_t pad = (1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u;
  float* ring = reinterpret_cast<float*>(smem_raw + pad);
  const int m1 = a.m1, m2 = a.m2, m3 = a.m3;
  const int bc = m2 * m3;
  float* s2 = ring + tc_block_ring_floats(2);  // m2 x m2
  float* s3 = s2 + al4(m2 * m2);              // m3 x m3
  float* ma = s3 + al4(m3 * m3);              // bc: M[a]
  float* wa = ma + al4(bc);                   // bc: W3[a], then scratch
  float* ga = wa + al4(bc);                   // bc: G[a]
  const int aa = blockIdx.x;
  const int64_t off = (int64_t)aa * bc;
  cp_flat(s2, a.S2, m2 * m2);
  cp_flat(wa, a.W3 + off, bc);
  cp_flat(ga, a.G + off, bc);
  cp_commit();
  const TcOperand As[2] = {{&map_y3, aa}, {nullptr, -1}};
  const TcOperand fb{&map_f3, -1};
  // M[a] rows b (m2 x m3, pitch m3) and S3 (m3 x m3, pitch m3).
  float* const outs[2] = {ma, s3};
  const int mss[2] = {m2, m3};
  const bool ok =
      tc_block_gemm<SPLIT, 2>(As, fb, (int)a.n3, ring, bars, outs, m3, mss, m3, a.err);
  cp_wait<0>();
  __syncthreads();
  if (!ok) return;
  if (aa == 0)
    for (int e = threadIdx.x; e < m3 * m3; e += blockDim.x) a.S3_out[e] = s3[e];
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {
    const int b = e / m3, c = e % m3;
    float d = 0.f;
    for (int w = 0; w < m3; ++w) d = fmaf(wa[b * m3 + w], s3[w * m3 + c], d);
    const float gv = mu_step(ga[e], ma[e], d, (float)a.eps);
    ga[e] = gv;
    a.G[off + e] = gv;
    a.G2[((int64_t)b * m1 + aa) * m3 + c] = gv;  // G permuted to (m2, m1, m3)
    a.G3[((int64_t)c * m1 + aa) * m2 + b] = gv;  // G permuted to (m3, m1, m2)
    a.Mout[off + e] = ma[e];
  }
  __syncthreads();
  smem_gemm(s2, ga, wa, m2, m2, m3);  // S2 G[a]
  __syncthreads();
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {  // W1[a] = (S2 G[a]) S3
    const int b = e / m3, c = e % m3;
    float v = 0.f;
    for (int w = 0; w < m3; ++w) v = fmaf(wa[b * m3 + w], s3[w * m3 + c], v);
    a.W1[off + e] = v;
  }
}

// ---------------------------------------------------------------------------
// core_b: one block per a: H1[a, q] = <W1[a], G[q]> (next sweep's H1) and
// <M[a], G[a]>. The residual also needs <G, G x_k S_k> = sum_{a,w} S1[a, w]
// H1[w, a] (Dn[a] = sum_w S1[a, w] W1[w], so <G[a], Dn[a]> = sum_w S1[a, w]
// <W1[w], G[a]>). The last block to finish adds the terms in a fixed order
// and writes the trace entry.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) core_b_kernel(CoreArgs<T> a) {
  if (a.gate && *a.gate == 0) return;  // no sweep since the last core update
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  __shared__ int last;
  const int m1 = a.m1, m2 = a.m2, m3 = a.m3;
  const int bc = m2 * m3;
  const bool gsm = core_in_smem<T>((int64_t)m1 * bc);
  T* wa = sm;             // bc: W1[a]
  T* gs = wa + al4(bc);   // m1 x bc when it fits
  const int aa = blockIdx.x;
  const int64_t off = (int64_t)aa * bc;
  cp_flat(wa, a.W1 + off, bc);
  if (gsm) cp_flat(gs, a.G, (int64_t)m1 * bc);
  cp_commit();
  double mg = 0.0;
  for (int e = threadIdx.x; e < bc; e += blockDim.x)
    mg += (double)a.Mout[off + e] * (double)a.G[off + e];
  cp_wait<0>();
  __syncthreads();
  mg = block_sum(mg, red);
  rows_dot(wa, gsm ? (const T*)gs : a.G, bc, m1, a.H1 + (int64_t)aa * m1);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.dots[aa] = mg;
    __threadfence();
    last = (atomicAdd(a.done, 1) == m1 - 1);
  }
  __syncthreads();
  if (!last) return;
  // Last block: every other block's H1 rows and dot are visible (fence +
  // atomic above); L2 loads (__ldcg) bypass this SM's L1.
  __threadfence();
  double pg = 0.0, pm = 0.0;
  for (int e = threadIdx.x; e < m1 * m1; e += blockDim.x) {
    const int r = e / m1, w = e % m1;
    pg += (double)a.S1[e] * (double)__ldcg(a.H1 + w * m1 + r);
  }
  for (int r = threadIdx.x; r < m1; r += blockDim.x) pm += __ldcg(a.dots + r);
  pg = block_sum(pg, red);
  pm = block_sum(pm, red);
  if (threadIdx.x == 0) {
    const double xx = *a.x2;
    double r2 = xx - 2.0 * pm + pg;
    const bool finite = isfinite(r2);
    if (r2 < 0.0) r2 = 0.0;
    trace_record(a.counter, a.trace, a.trace_stride, sqrt(r2 / xx), finite);
    *a.done = 0;  // ready for the next sweep
    if (a.gate) *a.gate = 0;
  }
}

// G2[b, a, c] = G[a, b, c], G3[c, a, b] = G[a, b, c] (the initial core).
template <typename T>
__global__ void permute_core_kernel(const T* __restrict__ G, int m1, int m2, int m3,
                                    T* __restrict__ G2, T* __restrict__ G3) {
  const int n = m1 * m2 * m3;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int c = e % m3, b = (e / m3) % m2, aa = e / (m2 * m3);
    G2[((int64_t)b * m1 + aa) * m3 + c] = G[e];
    G3[((int64_t)c * m1 + aa) * m2 + b] = G[e];
  }
}

// out[(k N2 + j) m1 + a] = in[(a N2 + j) N3 + k]: block (k tile of 32, j).
template <typename T>
__global__ void p1_rows_kernel(const T* __restrict__ in, int m1, int64_t N2, int64_t N3,
                               T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);  // m1 x 33
  const int64_t k0 = (int64_t)blockIdx.x * 32;
  for (int64_t j = blockIdx.y; j < N2; j += gridDim.y) {
    for (int e = threadIdx.x; e < m1 * 32; e += blockDim.x) {
      const int aa = e / 32, kk = e % 32;
      if (k0 + kk < N3) tile[aa * 33 + kk] = in[((int64_t)aa * N2 + j) * N3 + k0 + kk];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m1 * 32; e += blockDim.x) {
      const int kk = e / m1, aa = e % m1;
      if (k0 + kk < N3) out[((k0 + kk) * N2 + j) * m1 + aa] = tile[aa * 33 + kk];
    }
    __syncthreads();
  }
}

// S = F^T F for the prologue (one block).
template <typename T>
__global__ void __launch_bounds__(kThreads) gram_kernel(const T* __restrict__ F, int64_t N, int m,
                                                        T* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* c = sm + gemm_stage_elems(m, m, (int)sizeof(T), (int)N);
  gemm_tn_block(F, m, m, F, m, m, (int)N, gemm_kch(m, m, (int)sizeof(T), (int)N), c, sm);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) S[e] = c[e];
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

namespace {
template <typename K>
int set_smem(K kernel, size_t bytes) {
  NNC_CUDA_TRY(raise_smem_limit((const void*)kernel, bytes));
  return NNC_OK;
}
}  // namespace

// The shapes updt_kernel takes: mu, mc <= 32, the contraction rows of Fc and
// of every P_r starting on 16-byte boundaries (the tensor maps' rule for
// their base and strides), coordinates within int, and a flag for a copy that
// does not arrive.
static bool updt_fits(const UpdArgs<float>& a) {
  const int ms = a.p_first ? a.mc : a.mu;
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return a.mu >= 1 && a.mc >= 1 && a.mu <= 32 && a.mc <= 32 && a.len >= 1 && a.nrows >= 1 &&
         a.nrows < (1LL << 31) && ms % 4 == 0 && a.prow % 4 == 0 && a.pstride % 4 == 0 &&
         a.prow > 0 && a.pstride > 0 && al16(a.P) && al16(a.Fc) && a.err != nullptr;
}

bool upd_tc_form(const UpdArgs<float>& a) {
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int UC = a.mu * a.mc;
  if (!a.tc || a.mu < 1 || a.mc < 1 || a.mu > 32 || a.mc > 32 || a.mv < 1 || a.mv > 32 ||
      (UC & 3) != 0 || a.nrows < 1 || !al16(a.Gn) || a.err == nullptr)
    return false;
  if (a.Ypart) return a.nparts >= 1 && al16(a.Ypart) && (!a.Yout || al16(a.Yout));
  return a.ybuf != nullptr && al16(a.ybuf) && updt_fits(a);
}

int launch_upd_gemm(const UpdArgs<float>& a, cudaStream_t s) {
  if (a.Ypart || !upd_tc_form(a)) return NNC_ERR_UNSUPPORTED;
  const size_t smem = sizeof(float) * updt_smem_floats(a.mu, a.mc);
  const unsigned grid = (unsigned)ceil_div(a.nrows, (int64_t)kTcRows);
  // Fc: (ms, len), row pitch ms; P: (mr, len, nrows), strides pstride, prow.
  const int ms = a.p_first ? a.mc : a.mu, mr = a.p_first ? a.mu : a.mc;
  CUtensorMap map_f, map_p;
  {
    const uint64_t dims[2] = {(uint64_t)ms, (uint64_t)a.len};
    const uint64_t strides[1] = {(uint64_t)ms * 4};
    const uint32_t box[2] = {32, (uint32_t)kTcKC};
    NNC_TRY(tma::encode_f32(&map_f, a.Fc, 2, dims, strides, box));
  }
  {
    const uint64_t dims[3] = {(uint64_t)mr, (uint64_t)a.len, (uint64_t)a.nrows};
    const uint64_t strides[2] = {(uint64_t)a.pstride * 4, (uint64_t)a.prow * 4};
    const uint32_t box[3] = {32, (uint32_t)kTcKC, (uint32_t)kTcRows};
    NNC_TRY(tma::encode_f32(&map_p, a.P, 3, dims, strides, box));
  }
  if (a.tc == 3) {
    NNC_TRY(set_smem(updt_kernel<3>, smem));
    updt_kernel<3><<<grid, kThreads, smem, s>>>(a, map_f, map_p);
  } else {
    NNC_TRY(set_smem(updt_kernel<1>, smem));
    updt_kernel<1><<<grid, kThreads, smem, s>>>(a, map_f, map_p);
  }
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

int launch_upd_num(const UpdArgs<float>& a, cudaStream_t s) {
  if (!upd_tc_form(a) || (a.num_only && !a.num)) return NNC_ERR_UNSUPPORTED;
  const size_t smem = sizeof(float) * numu_smem_floats(a.mu, a.mc, a.mv);
  const unsigned grid = (unsigned)ceil_div(a.nrows, (int64_t)kNuRows);
  if (a.tc == 3) {
    NNC_TRY(set_smem(numu_kernel<3>, smem));
    NNC_CUDA_TRY(launch_pdl(numu_kernel<3>, dim3(grid), dim3(kNuThreads), smem, s, a));
  } else {
    NNC_TRY(set_smem(numu_kernel<1>, smem));
    NNC_CUDA_TRY(launch_pdl(numu_kernel<1>, dim3(grid), dim3(kNuThreads), smem, s, a));
  }
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_upd12(const UpdArgs<T>& a, cudaStream_t s) {
  if (a.mu > 64 || a.mc > 64 || a.mv > 64) return NNC_ERR_UNSUPPORTED;
  const int UC = a.mu * a.mc;
  if constexpr (std::is_same<T, float>::value) {
    if (upd_tc_form(a)) {
      if (!a.Ypart) NNC_TRY(launch_upd_gemm(a, s));
      return launch_upd_num(a, s);
    }
  }
  if (a.Ypart) {
    const size_t smem = sizeof(T) * (al4((size_t)2 * UC) + al4((size_t)a.mv * a.mv) +
                                     2 * al4((size_t)2 * a.mv));
    NNC_TRY(set_smem(upds_kernel<T>, smem));
    upds_kernel<T><<<(unsigned)ceil_div(a.nrows, (int64_t)2), kThreads, smem, s>>>(a);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  }
  {
    // The GEMM form: R rows per block (updm_kernel).
    const int R = Updm<T>::rows(a.mu, a.mc);
    const size_t smem = sizeof(T) * Updm<T>::stage_elems(a.mu, a.mc, a.mv, a.p_first, nullptr);
    NNC_TRY(set_smem(updm_kernel<T>, smem));
    updm_kernel<T><<<(unsigned)ceil_div(a.nrows, (int64_t)R), kThreads, smem, s>>>(a);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  }
}

template <typename T>
int launch_mu_rows(const UpdArgs<T>& a, cudaStream_t s) {
  if (a.mv > 64 || a.mv < 1 || !a.num) return NNC_ERR_UNSUPPORTED;
  const int R = kThreads / a.mv;
  const size_t smem = sizeof(T) * (al4(a.mv * a.mv) + al4((size_t)R * a.mv));
  NNC_TRY(set_smem(mu_rows_kernel<T>, smem));
  mu_rows_kernel<T><<<(unsigned)ceil_div(a.nrows, (int64_t)R), kThreads, smem, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

static bool al16p(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// hmat_tc_kernel's shapes: one Gram to form (fu or fv), every dimension <=
// 32, the factor's rows 16-byte aligned.
static bool hmat_tc_fits(const HArgs<float>& a) {
  if (!a.tc || !a.err || (a.fu != nullptr) == (a.fv != nullptr)) return false;
  const float* f = a.fu ? a.fu : a.fv;
  const int m = a.fu ? a.mu : a.mv;
  const int64_t n = a.fu ? a.nu : a.nv;
  return a.mp >= 1 && a.mp <= 32 && a.mu >= 1 && a.mu <= 32 && a.mv >= 1 && a.mv <= 32 &&
         m % 4 == 0 && n >= 1 && n < (1LL << 31) && al16p(f);
}

template <typename T>
int launch_hmat(const HArgs<T>& a, cudaStream_t s) {
  if (a.mu > 64 || a.mv > 64) return NNC_ERR_UNSUPPORTED;
  if constexpr (std::is_same<T, float>::value) {
    if (hmat_tc_fits(a)) {
      const int m = a.fu ? a.mu : a.mv;
      const uint64_t dims[2] = {(uint64_t)m, (uint64_t)(a.fu ? a.nu : a.nv)};
      const uint64_t strides[1] = {(uint64_t)m * 4};
      const uint32_t box[2] = {32, 64};
      CUtensorMap map_f;
      NNC_TRY(tma::encode_f32(&map_f, a.fu ? a.fu : a.fv, 2, dims, strides, box));
      const size_t smem = sizeof(float) * (256 + tc_block_ring_floats(1) + al4(a.mu * a.mu) +
                                           al4(a.mv * a.mv) + 3 * al4(a.mu * a.mv));
      if (a.tc == 3) {
        NNC_TRY(set_smem(hmat_tc_kernel<3>, smem));
        hmat_tc_kernel<3><<<a.mp, kThreads, smem, s>>>(a, map_f);
      } else {
        NNC_TRY(set_smem(hmat_tc_kernel<1>, smem));
        hmat_tc_kernel<1><<<a.mp, kThreads, smem, s>>>(a, map_f);
      }
      note_launch(s);
      NNC_CUDA_TRY(cudaGetLastError());
      return NNC_OK;
    }
  }
  const size_t st_u = a.fu ? gemm_stage_elems(a.mu, a.mu, (int)sizeof(T), (int)a.nu) : 0;
  const size_t st_v = a.fv ? gemm_stage_elems(a.mv, a.mv, (int)sizeof(T), (int)a.nv) : 0;
  const int64_t guv = (int64_t)a.mp * a.mu * a.mv;
  const size_t smem = sizeof(T) * ((st_u > st_v ? st_u : st_v) + al4(a.mu * a.mu) +
                                   al4(a.mv * a.mv) + 3 * al4(a.mu * a.mv) +
                                   (core_in_smem<T>(guv) ? (size_t)guv : 0));
  NNC_TRY(set_smem(hmat_kernel<T>, smem));
  hmat_kernel<T><<<a.mp, kThreads, smem, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_p1_rows(const T* in, int m1, int64_t N2, int64_t N3, T* out, cudaStream_t s) {
  if (m1 > 64) return NNC_ERR_UNSUPPORTED;
  const size_t smem = sizeof(T) * (size_t)m1 * 33;
  NNC_TRY(set_smem(p1_rows_kernel<T>, smem));
  dim3 grid((unsigned)ceil_div(N3, 32), (unsigned)(N2 < 65535 ? N2 : 65535));
  p1_rows_kernel<T><<<grid, kThreads, smem, s>>>(in, m1, N2, N3, out);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

// core_a_tc_kernel's shapes: every m <= 32, m2 and m3 multiples of 4 (the
// rows of F3 and Y3 16-byte aligned).
static bool core_tc_fits(const CoreArgs<float>& a) {
  return a.tc && a.err && a.m1 >= 1 && a.m1 <= 32 && a.m2 >= 4 && a.m2 <= 32 && a.m3 >= 4 &&
         a.m3 <= 32 && a.m2 % 4 == 0 && a.m3 % 4 == 0 && a.n3 >= 1 && a.n3 < (1LL << 31) &&
         al16p(a.F3) && al16p(a.Y3);
}

template <typename T>
int launch_core(const CoreArgs<T>& a, cudaStream_t s) {
  if (a.m1 > 64 || a.m2 > 64 || a.m3 > 64) return NNC_ERR_UNSUPPORTED;
  const int bc = a.m2 * a.m3;
  bool tc_done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (core_tc_fits(a)) {
      CUtensorMap map_f3, map_y3;
      {
        const uint64_t dims[2] = {(uint64_t)a.m3, (uint64_t)a.n3};
        const uint64_t strides[1] = {(uint64_t)a.m3 * 4};
        const uint32_t box[2] = {32, 64};
        NNC_TRY(tma::encode_f32(&map_f3, a.F3, 2, dims, strides, box));
      }
      {  // Y3 laid out (N3, m1, m2): entry (b, k, a) of the map
        const uint64_t dims[3] = {(uint64_t)a.m2, (uint64_t)a.n3, (uint64_t)a.m1};
        const uint64_t strides[2] = {(uint64_t)a.m1 * a.m2 * 4, (uint64_t)a.m2 * 4};
        const uint32_t box[3] = {32, 64, 1};
        NNC_TRY(tma::encode_f32(&map_y3, a.Y3, 3, dims, strides, box));
      }
      const size_t smem = sizeof(float) * (256 + tc_block_ring_floats(2) + al4(a.m2 * a.m2) +
                                           al4(a.m3 * a.m3) + 3 * al4(bc));
      if (a.tc == 3) {
        NNC_TRY(set_smem(core_a_tc_kernel<3>, smem));
        core_a_tc_kernel<3><<<a.m1, kThreads, smem, s>>>(a, map_f3, map_y3);
      } else {
        NNC_TRY(set_smem(core_a_tc_kernel<1>, smem));
        core_a_tc_kernel<1><<<a.m1, kThreads, smem, s>>>(a, map_f3, map_y3);
      }
      note_launch(s);
      NNC_CUDA_TRY(cudaGetLastError());
      tc_done = true;
    }
  }
  if (!tc_done) {
    const size_t st3 = gemm_stage_elems(a.m3, a.m3, (int)sizeof(T), (int)a.n3);
    const size_t stm = gemm_stage_elems(a.m2, a.m3, (int)sizeof(T), (int)a.n3);
    const size_t smem_a = sizeof(T) * ((st3 > stm ? st3 : stm) + al4(a.m2 * a.m2) +
                                       al4(a.m3 * a.m3) + 3 * al4(bc));
    NNC_TRY(set_smem(core_a_kernel<T>, smem_a));
    core_a_kernel<T><<<a.m1, kThreads, smem_a, s>>>(a);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
  }
  const int64_t g = (int64_t)a.m1 * bc;
  const size_t smem_b = sizeof(T) * (al4(bc) + (core_in_smem<T>(g) ? (size_t)g : 0));
  NNC_TRY(set_smem(core_b_kernel<T>, smem_b));
  core_b_kernel<T><<<a.m1, kThreads, smem_b, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_gram(const T* F, int64_t N, int m, T* S, cudaStream_t s) {
  if (m > 64) return NNC_ERR_UNSUPPORTED;
  const size_t smem =
      sizeof(T) * (gemm_stage_elems(m, m, (int)sizeof(T), (int)N) + al4((size_t)m * m));
  NNC_TRY(set_smem(gram_kernel<T>, smem));
  gram_kernel<T><<<1, kThreads, smem, s>>>(F, N, m, S);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_permute_core(const T* G, int m1, int m2, int m3, T* G2, T* G3, cudaStream_t s) {
  const int n = m1 * m2 * m3;
  permute_core_kernel<T><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(G, m1, m2, m3, G2, G3);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

#define NNC_SWEEP_INST(T)                                                                   \
  template int launch_upd12<T>(const UpdArgs<T>&, cudaStream_t);                            \
  template int launch_hmat<T>(const HArgs<T>&, cudaStream_t);                               \
  template int launch_mu_rows<T>(const UpdArgs<T>&, cudaStream_t);                          \
  template int launch_p1_rows<T>(const T*, int, int64_t, int64_t, T*, cudaStream_t);       \
  template int launch_core<T>(const CoreArgs<T>&, cudaStream_t);                            \
  template int launch_gram<T>(const T*, int64_t, int, T*, cudaStream_t);                    \
  template int launch_permute_core<T>(const T*, int, int, int, T*, T*, cudaStream_t);
NNC_SWEEP_INST(float)
NNC_SWEEP_INST(double)
#undef NNC_SWEEP_INST

}  // namespace nnc
