// Fused kernels of one nnTD sweep around the two passes over X.
//
// With P3 = X x_3 F3^T ((N1 N2) x m3) and P1 = X x_1 F1^T (rows (k, j) x m1)
// from the passes, a sweep is (S_k = F_k^T F_k, Eq. unfolding:property):
//
//   upd12 (mode 1) per slab i:  Y1[i] = F2^T P3[i, :, :]           (m2 x m3)
//                               (or the sum of its shares formed by pass 1)
//                               Num1[i, a] = <Y1[i], G[a, :, :]>
//                               F1[i, :] <- MU with Den = F1[i, :] H1
//   hmat  (mode 2) per b:       S1 = F1^T F1;  W[:, b, :] = S1 G[:, b, :] S3
//                               H2[b, b'] = <W[:, b, :], G[:, b', :]>
//   upd12 (mode 2) per row j:   Y2[:, j, :] = F1^T P3[:, j, :];  Num2 (numerator only)
//   mu_rows (mode 2):           MU on F2 with Den = F2 H2
//   hmat  (mode 3) per c:       S2 = F2^T F2;  W3 = G x_1 S1 x_2 S2 (kept);  H3
//   upd12 (mode 3) per slab k:  Y3[k] = P1[k, :, :]^T F2  (m1 x m2, kept)
//                               (or the sum of its shares formed by pass 2)
//                               Num3[k, c] = <Y3[k], G[:, :, c]>;  MU on F3
//   core_a (one block per a):   S3 = F3^T F3; M[a] = Y3[:, a, :]^T F3 (= (X x_1 F1^T x_2 F2^T x_3 F3^T)[a]);
//                               D = W3 x_3 S3;  G <- MU(G, M, D); W1 = G x_2 S2 x_3 S3
//   core_b (one block per a):   H1 = unfold_1(W1) unfold_1(G)^T for the next sweep;
//                               trace = sqrt(||X||^2 - 2<M,G> + <G, G x_k S_k>)/||X||
//                               with <G, G x_k S_k> = sum S1 .* H1^T (last block)
//
// These kernels are latency-bound (a few MFLOP each on L2-resident data), so
// each block requests everything it needs up front (cp.async) and spreads every
// contraction over all its threads: the block GEMM splits the contraction
// across thread groups (4 x 4 register tiles per thread). Most blocks run
// their code once per sweep with a cold instruction cache, so the shared
// helpers are kept out of line and not unrolled (one copy of the code per
// kernel). Every reduction runs in a fixed order, so results are
// deterministic. The BF16 path also writes, from the mode-1 and mode-3
// updates, the BF16 operand of the next pass over X.
#include <cuda_bf16.h>

#include <type_traits>

#include "kernels.cuh"
#include "sweep.cuh"

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
// NS partial sums are added by a fixed shuffle tree.
template <typename T>
__device__ __noinline__ void rows_dot2(const T* x0, const T* x1, const T* Y, int n, int nq,
                                       T* out0, T* out1) {
  const int NS = nq > 32 ? 4 : 8;
  const int per = blockDim.x / NS;  // rows at a time
  const int s = threadIdx.x % NS;
  const bool vec = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
  for (int q0 = 0; q0 < nq; q0 += per) {
    const int q = q0 + threadIdx.x / NS;
    T a0 = T(0), a1 = T(0);
    if (q < nq) {
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
    if (q < nq && s == 0) {
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

// ---------------------------------------------------------------------------
// upd12: factor update of one mode from a pass result, one block per row r.
//   Y_r = Fc^T P_r or P_r^T Fc (mu x mc), or the sum of its shares that the
//   pass already formed;  Num[r, v] = <Y_r, Gn[v]>;
//   F[r] <- MU(F[r], Num, F[r] H)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) upd12_kernel(UpdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MU_ = a.mu, MC = a.mc, MV = a.mv, UC = MU_ * MC;
  const bool gsm = core_in_smem<T>((int64_t)MV * UC);
  T* stage = sm;
  T* ys = stage + (a.Ypart ? 0 : gemm_stage_elems(MU_, MC, (int)sizeof(T), a.len));
  T* hs = ys + al4(UC);
  T* fo = hs + al4(MV * MV);
  T* nm = fo + al4(MV);
  T* gs = nm + al4(MV);  // MV x UC when it fits
  const int64_t r = blockIdx.x;
  // A programmatic successor (the next sweep's first pass over X) may start
  // its prologue and its reads of X now; it waits for this grid before it
  // reads anything this kernel writes.
  pdl_trigger();

  // Everything but the GEMM operands is requested first; the GEMM's waits
  // cover this group too.
  if (!a.num_only) {
    cp_flat(hs, a.H, MV * MV);
    cp_flat(fo, a.F + r * MV, MV);
  }
  if (gsm) cp_flat(gs, a.Gn, (int64_t)MV * UC);
  cp_commit();
  if (a.Ypart) {
    const T* yp = a.Ypart + r * a.nparts * UC;
    for (int e = threadIdx.x; e < UC; e += blockDim.x) {
      T y = yp[e];
      for (int h = 1; h < a.nparts; ++h) y += yp[(int64_t)h * UC + e];
      ys[e] = y;
    }
    cp_wait<0>();
    __syncthreads();
  } else {
    const int kch = gemm_kch(MU_, MC, (int)sizeof(T), a.len);
    const T* pr = a.P + r * a.prow;
    if (a.p_first)
      gemm_tn_block(pr, a.pstride, MU_, a.Fc, MC, MC, a.len, kch, ys, stage);
    else
      gemm_tn_block(a.Fc, MU_, MU_, pr, a.pstride, MC, a.len, kch, ys, stage);
  }

  if (a.Yout)
    for (int e = threadIdx.x; e < UC; e += blockDim.x) a.Yout[r * UC + e] = ys[e];
  if (a.num_only) {
    rows_dot(ys, gsm ? (const T*)gs : a.Gn, UC, MV, a.num + r * MV);
    return;
  }
  rows_dot(ys, gsm ? (const T*)gs : a.Gn, UC, MV, nm);
  __syncthreads();
  for (int v = threadIdx.x; v < MV; v += blockDim.x) {
    T den = T(0);
    for (int w = 0; w < MV; ++w) den = fma(fo[w], hs[w * MV + v], den);
    const T nv = mu_step(fo[v], nm[v], den, (T)a.eps);
    a.F[r * MV + v] = nv;
    write_operand(a, r, v, nv);
  }
  if (a.gate_out && r == 0 && threadIdx.x == 0) *a.gate_out = 1;
}

// ---------------------------------------------------------------------------
// updm: the update of upd12 for R rows per block, the GEMMs staged by a
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
  pdl_trigger();  // as in upd12

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
  if (a.Yout)
    for (int e = threadIdx.x; e < rn * UC; e += blockDim.x) a.Yout[r0 * UC + e] = ys[e];
  // Numerators of the R rows, each core row read once for the block.
  if (a.num_only) {
    rows_dot2<T>(ys, R > 1 ? ys + UC : nullptr, a.Gn, UC, MV, nm, nm + MV);
    __syncthreads();
    for (int e = threadIdx.x; e < rn * MV; e += blockDim.x) a.num[r0 * MV + e] = nm[e];
    return;
  }
  rows_dot2<T>(ys, R > 1 ? ys + UC : nullptr, a.Gn, UC, MV, nm, nm + MV);
  __syncthreads();
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
// mu_rows: the MU step of a split update, kThreads / mv rows per block.
//   F[r, v] <- MU(F[r, v], num[r, v], sum_w F[r, w] H[w, v])
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) mu_rows_kernel(UpdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MV = a.mv, R = kThreads / MV;
  pdl_trigger();  // as in upd12
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

template <typename T>
int launch_upd12(const UpdArgs<T>& a, cudaStream_t s) {
  if (a.mu > 64 || a.mc > 64 || a.mv > 64) return NNC_ERR_UNSUPPORTED;
  const int UC = a.mu * a.mc;
  if (!a.Ypart) {
    // The GEMM form: R rows per block (updm_kernel).
    const int R = Updm<T>::rows(a.mu, a.mc);
    const size_t smem = sizeof(T) * Updm<T>::stage_elems(a.mu, a.mc, a.mv, a.p_first, nullptr);
    NNC_TRY(set_smem(updm_kernel<T>, smem));
    updm_kernel<T><<<(unsigned)ceil_div(a.nrows, (int64_t)R), kThreads, smem, s>>>(a);
    note_launch(s);
    NNC_CUDA_TRY(cudaGetLastError());
    return NNC_OK;
  }
  const size_t st = a.Ypart ? 0 : gemm_stage_elems(a.mu, a.mc, (int)sizeof(T), a.len);
  const size_t smem =
      sizeof(T) * (st + al4(UC) + al4(a.mv * a.mv) + 2 * al4(a.mv) +
                   (core_in_smem<T>((int64_t)a.mv * UC) ? (size_t)a.mv * UC : 0));
  NNC_TRY(set_smem(upd12_kernel<T>, smem));
  upd12_kernel<T><<<(unsigned)a.nrows, kThreads, smem, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
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

template <typename T>
int launch_hmat(const HArgs<T>& a, cudaStream_t s) {
  if (a.mu > 64 || a.mv > 64) return NNC_ERR_UNSUPPORTED;
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

template <typename T>
int launch_core(const CoreArgs<T>& a, cudaStream_t s) {
  if (a.m1 > 64 || a.m2 > 64 || a.m3 > 64) return NNC_ERR_UNSUPPORTED;
  const int bc = a.m2 * a.m3;
  const size_t st3 = gemm_stage_elems(a.m3, a.m3, (int)sizeof(T), (int)a.n3);
  const size_t stm = gemm_stage_elems(a.m2, a.m3, (int)sizeof(T), (int)a.n3);
  const size_t smem_a = sizeof(T) * ((st3 > stm ? st3 : stm) + al4(a.m2 * a.m2) +
                                     al4(a.m3 * a.m3) + 3 * al4(bc));
  NNC_TRY(set_smem(core_a_kernel<T>, smem_a));
  core_a_kernel<T><<<a.m1, kThreads, smem_a, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
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
