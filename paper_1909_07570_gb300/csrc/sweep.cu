// Fused kernels of one nnTD sweep around the two passes over X.
//
// With P3 = X x_3 F3^T ((N1 N2) x m3) and P1 = X x_1 F1^T (m1 x N2 x N3) from
// the passes, a sweep is (S_k = F_k^T F_k, Eq. unfolding:property):
//
//   upd12 (mode 1) per slab i:  Y1[i] = F2^T P3[i, :, :]           (m2 x m3)
//                               Num1[i, a] = <Y1[i], G[a, :, :]>
//                               F1[i, :] <- MU with Den = F1[i, :] H1
//   hmat  (mode 2) per b:       S1 = F1^T F1;  W[:, b, :] = S1 G[:, b, :] S3
//                               H2[b, b'] = <W[:, b, :], G[:, b', :]>
//   upd12 (mode 2) per row j:   Y2[:, j, :] = F1^T P3[:, j, :];  Num2;  MU on F2
//   hmat  (mode 3) per c:       S2 = F2^T F2;  W3 = G x_1 S1 x_2 S2 (kept);  H3
//   y3:                         Y3[a, b, k] = sum_j P1[a, j, k] F2[j, b]
//   num3 + tail3:               Num3[k, c] = sum_{a,b} Y3[a, b, k] G[a, b, c] (split over
//                               (a, b), added in split order); MU on F3
//   core_m:                     M = Y3 x_3 F3^T (split over k)
//   core_a (one block per a):   S3 = F3^T F3; D = W3 x_3 S3; G <- MU(G, M, D);
//                               W1 = G x_2 S2 x_3 S3
//   core_b (one block per a):   H1 = unfold_1(W1) unfold_1(G)^T for the next sweep;
//                               trace = sqrt(||X||^2 - 2<M,G> + <G, G x_k S_k>)/||X||
//                               with <G, G x_k S_k> = sum S1 .* H1^T (last block)
//
// The contractions are SIMT GEMMs on 4 x 4 register tiles whose operands are
// staged in shared memory by cp.async, two chunks in flight. Every reduction
// runs in a fixed order, so results are deterministic. The BF16 path also
// writes, from the mode-1 and mode-3 updates, the BF16 operand of the next
// pass over X.
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
      const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);  // exact TF32 part
      uint32_t l;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - h));
      a.bhi[idx] = h;
      a.blo[idx] = __uint_as_float(l);
    }
  }
}

template <typename T>
__device__ __forceinline__ T mu_step(T theta, T num, T den, T eps) {
  const T v = theta * num / (den > eps ? den : eps);
  return v > T(0) ? v : T(0);
}

// ---- cp.async staging (element granularity, zero fill outside the range) ----
template <typename T>
__device__ __forceinline__ void cp_elem(T* dst, const T* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 16-byte cp.async of one vector (16 / sizeof(T) elements); the first `valid`
// elements are copied, the rest of the vector is zero.
template <typename T>
__device__ __forceinline__ void cp_vec(T* dst, const T* src, int valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int n = valid * (int)sizeof(T);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n)
               : "memory");
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

// acc[i][j] += sum_{k < kn} A[k][m0 + i] B[k][n0 + j]
template <typename T>
__device__ __forceinline__ void tile4x4(const T* A, int lda, const T* B, int ldb, int kn, int m0,
                                        int n0, T (&acc)[4][4]) {
  for (int k = 0; k < kn; ++k) {
    T a[4], b[4];
    ld4(A + k * lda + m0, a);
    ld4(B + k * ldb + n0, b);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

template <typename T>
__device__ __forceinline__ void zero4x4(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}

// Rows of F staged per chunk by gram_block: up to 32 KB of shared memory.
__host__ __device__ constexpr int gram_rows(int m, int elem) {
  return (32 * 1024) / (r4(m) * elem) < 1 ? 1 : (32 * 1024) / (r4(m) * elem);
}

// S = F^T F (n rows of width m) into shared s (m x m), computed by the whole
// block: groups of threads take interleaved rows with 4 x 4 tiles of S and are
// added in group order. F is staged by cp.async in chunks of gram_rows rows;
// `stage` holds gram_stage_elems(m) elements (chunk + per-group partials).
template <typename T>
__device__ void gram_block(const T* __restrict__ F, int64_t n, int m, T* s, T* stage) {
  const int mq = r4(m) / 4, tiles = mq * mq;
  const int groups = max(1, (int)blockDim.x / tiles);
  const int g = threadIdx.x / tiles, t = threadIdx.x % tiles;
  const int x0 = (t / mq) * 4, y0 = (t % mq) * 4;
  const int RC = gram_rows(m, (int)sizeof(T));
  T* fs = stage;                             // RC x r4(m)
  T* red = stage + al4((size_t)RC * r4(m));  // groups x m x m
  T acc[4][4];
  zero4x4(acc);
  for (int64_t r0 = 0; r0 < n; r0 += RC) {
    const int rn = (int)((n - r0) < (int64_t)RC ? (n - r0) : (int64_t)RC);
    stage_tile(fs, r4(m), F + r0 * m, m, rn, r4(m), rn, m, aligned16(F + r0 * m, m, sizeof(T)));
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    if (g < groups) {
      for (int rr = g; rr < rn; rr += groups) {
        T a[4], b[4];
        ld4(fs + rr * r4(m) + x0, a);
        ld4(fs + rr * r4(m) + y0, b);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (g < groups) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (x0 + i < m && y0 + j < m) red[(g * m + x0 + i) * m + y0 + j] = acc[i][j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    T v = T(0);
    for (int q = 0; q < groups; ++q) v += red[q * m * m + e];
    s[e] = v;
  }
  __syncthreads();
}

// sum_e x[e] y[e] over e = lane, lane + 32, ... < n, then over the warp.
template <typename T>
__device__ __forceinline__ T warp_dot(const T* x, const T* __restrict__ y, int n, int lane) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int e = lane;
  for (; e + 96 < n; e += 128) {
    s0 = fma(x[e], y[e], s0);
    s1 = fma(x[e + 32], y[e + 32], s1);
    s2 = fma(x[e + 64], y[e + 64], s2);
    s3 = fma(x[e + 96], y[e + 96], s3);
  }
  for (; e < n; e += 32) s0 = fma(x[e], y[e], s0);
  return warp_sum((s0 + s1) + (s2 + s3));
}

// ---------------------------------------------------------------------------
// upd12: factor update of mode 1 or 2 from P3.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) upd12_kernel(UpdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MU_ = a.mu, MC = a.mc, MV = a.mv, S = a.rows_per_block;
  const int mu4 = r4(MU_), mc4 = r4(MC);
  const int tiles = (mu4 / 4) * (mc4 / 4);
  T* As = sm;                          // 2 x KC x mu4
  T* Bs = As + 2 * KC * mu4;           // 2 x S x KC x mc4
  T* ys = Bs + 2 * S * KC * mc4;       // S x MU_ x MC
  T* fo = ys + S * MU_ * MC;           // S x MV
  T* hs = fo + S * MV;                 // MV x MV
  T* nm = hs + MV * MV;                // S x MV
  const int64_t r0 = (int64_t)blockIdx.x * S;

  for (int e = threadIdx.x; e < MV * MV; e += blockDim.x) hs[e] = a.H[e];
  for (int e = threadIdx.x; e < S * MV; e += blockDim.x) {
    const int rr = e / MV, v = e % MV;
    fo[e] = (r0 + rr < a.nrows) ? a.F[(r0 + rr) * MV + v] : T(0);
  }

  const int nchunks = (a.len + KC - 1) / KC;
  const bool vecA = aligned16(a.Fc, MU_, sizeof(T));
  const bool vecB = aligned16(a.P, a.prow, sizeof(T)) && aligned16(a.P, a.pstride, sizeof(T));
  auto issue = [&](int c, int buf) {
    const int t0 = c * KC;
    const int tn = min(KC, a.len - t0);
    T* A = As + buf * KC * mu4;
    T* B = Bs + buf * S * KC * mc4;
    stage_tile(A, mu4, a.Fc + (int64_t)t0 * MU_, MU_, KC, mu4, tn, MU_, vecA);
    for (int rr = 0; rr < S; ++rr) {
      const int64_t r = r0 + rr;
      stage_tile(B + rr * KC * mc4, mc4, a.P + (r < a.nrows ? r : 0) * a.prow +
                 (int64_t)t0 * a.pstride, a.pstride, KC, mc4, r < a.nrows ? tn : 0, MC, vecB);
    }
    cp_commit();
  };

  const int my_s = threadIdx.x / tiles, my_t = threadIdx.x % tiles;
  const bool act = my_s < S;
  const int u0 = (my_t / (mc4 / 4)) * 4, c0 = (my_t % (mc4 / 4)) * 4;
  T acc[4][4];
  zero4x4(acc);
  issue(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1, (c + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (act) {
      const int kn = min(KC, a.len - c * KC);
      tile4x4(As + (c & 1) * KC * mu4, mu4, Bs + (c & 1) * S * KC * mc4 + my_s * KC * mc4, mc4,
              kn, u0, c0, acc);
    }
    __syncthreads();
  }
  if (act) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (u0 + i < MU_ && c0 + j < MC) ys[(my_s * MU_ + u0 + i) * MC + c0 + j] = acc[i][j];
  }
  __syncthreads();

  // Num[r, v] = <Y_r, Gn[v, :]>: one warp per (r, v); Gn rows are contiguous.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int UC = MU_ * MC;
  for (int task = warp; task < S * MV; task += nw) {
    const int rr = task / MV, v = task % MV;
    const T s = warp_dot(ys + rr * UC, a.Gn + (int64_t)v * UC, UC, lane);
    if (lane == 0) nm[task] = s;
  }
  __syncthreads();

  // MU with Den = F_old H; BF16 operand of the next pass if requested.
  for (int e = threadIdx.x; e < S * MV; e += blockDim.x) {
    const int rr = e / MV, v = e % MV;
    const int64_t r = r0 + rr;
    if (r >= a.nrows) continue;
    T den = T(0);
    for (int w = 0; w < MV; ++w) den = fma(fo[rr * MV + w], hs[w * MV + v], den);
    const T nv = mu_step(fo[e], nm[e], den, (T)a.eps);
    a.F[r * MV + v] = nv;
    write_operand(a, r, v, nv);
  }
}

// ---------------------------------------------------------------------------
// hmat: H_n for one mode (and optionally the W slices), one block per p.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) hmat_kernel(HArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int U = a.mu, V = a.mv, P = a.mp;
  T* su = sm;                  // U x U
  T* sv = su + al4(U * U);     // V x V
  T* gp = sv + al4(V * V);     // U x V
  T* tp = gp + al4(U * V);     // U x V
  T* wp = tp + al4(U * V);     // U x V
  T* stage = wp + al4(U * V);  // Gram staging
  const int p = blockIdx.x;
  if (a.fu) {
    gram_block(a.fu, a.nu, U, su, stage);
  } else {
    for (int e = threadIdx.x; e < U * U; e += blockDim.x) su[e] = a.su[e];
  }
  if (a.fv) {
    gram_block(a.fv, a.nv, V, sv, stage);
  } else {
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) sv[e] = a.sv[e];
  }
  for (int e = threadIdx.x; e < U * V; e += blockDim.x) gp[e] = a.Gn[(int64_t)p * U * V + e];
  __syncthreads();
  if (p == 0 && a.su_out && a.fu)
    for (int e = threadIdx.x; e < U * U; e += blockDim.x) a.su_out[e] = su[e];
  if (p == 0 && a.sv_out && a.fv)
    for (int e = threadIdx.x; e < V * V; e += blockDim.x) a.sv_out[e] = sv[e];
  for (int e = threadIdx.x; e < U * V; e += blockDim.x) {  // tp = S_u gp
    const int u = e / V, v = e % V;
    T s = T(0);
    for (int w = 0; w < U; ++w) s = fma(su[u * U + w], gp[w * V + v], s);
    tp[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < U * V; e += blockDim.x) {  // wp = tp S_v
    const int u = e / V, v = e % V;
    T s = T(0);
    for (int w = 0; w < V; ++w) s = fma(tp[u * V + w], sv[w * V + v], s);
    wp[e] = s;
    if (a.Wout) a.Wout[(int64_t)p * a.w_sp + (int64_t)u * a.w_su + (int64_t)v * a.w_sv] = s;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < P; q += kThreads / 32) {  // H[p, q] = <wp, G_q>
    const T s = warp_dot(wp, a.Gn + (int64_t)q * U * V, U * V, lane);
    if (lane == 0) a.H[p * P + q] = s;
  }
}

// ---------------------------------------------------------------------------
// y3: Y3[a, b, k] = sum_j P1[a, j, k] F2[j, b]; block (k tile of 64, a).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) y3_kernel(const T* __restrict__ P1,
                                                      const T* __restrict__ F2, int N2, int N3,
                                                      int m2, T* __restrict__ Y3) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int MT = 64;
  const int m24 = r4(m2);
  T* As = sm;                   // 2 x KC x MT
  T* Bs = As + 2 * KC * MT;     // 2 x KC x m24
  const int ai = blockIdx.y, k0 = blockIdx.x * MT;
  const T* p1 = P1 + (int64_t)ai * N2 * N3;
  const int nchunks = (N2 + KC - 1) / KC;
  const bool vecA = aligned16(p1 + k0, N3, sizeof(T));
  const bool vecB = aligned16(F2, m2, sizeof(T));
  auto issue = [&](int c, int buf) {
    const int j0 = c * KC;
    const int jn = min(KC, N2 - j0);
    stage_tile(As + buf * KC * MT, MT, p1 + (int64_t)j0 * N3 + k0, N3, KC, MT, jn, N3 - k0, vecA);
    stage_tile(Bs + buf * KC * m24, m24, F2 + (int64_t)j0 * m2, m2, KC, m24, jn, m2, vecB);
    cp_commit();
  };
  const int tiles = (MT / 4) * (m24 / 4);
  const bool act = threadIdx.x < tiles;
  const int kq = (threadIdx.x % (MT / 4)) * 4, bq = (threadIdx.x / (MT / 4)) * 4;
  T acc[4][4];
  zero4x4(acc);
  issue(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1, (c + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (act)
      tile4x4(As + (c & 1) * KC * MT, MT, Bs + (c & 1) * KC * m24, m24, min(KC, N2 - c * KC), kq,
              bq, acc);
    __syncthreads();
  }
  if (act) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = bq + j;
      if (b >= m2) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = k0 + kq + i;
        if (k < N3) Y3[((int64_t)ai * m2 + b) * N3 + k] = acc[i][j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// num3: part[s][k][c] = sum_{u in split s} Y3[u, k] G[u, c]; block (k tile, split).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) num3_kernel(const T* __restrict__ Y3,
                                                        const T* __restrict__ G, int UC, int N3,
                                                        int m3, int u_per_split,
                                                        T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int MT = 64;
  const int m34 = r4(m3);
  T* As = sm;
  T* Bs = As + 2 * KC * MT;
  const int k0 = blockIdx.x * MT;
  const int ub = blockIdx.y * u_per_split, ue = min(UC, ub + u_per_split);
  const int nchunks = (ue - ub + KC - 1) / KC;
  const bool vecA = aligned16(Y3 + k0, N3, sizeof(T));
  const bool vecB = aligned16(G, m3, sizeof(T));
  auto issue = [&](int c, int buf) {
    const int u0 = ub + c * KC;
    const int un = min(KC, ue - u0);
    stage_tile(As + buf * KC * MT, MT, Y3 + (int64_t)u0 * N3 + k0, N3, KC, MT, un, N3 - k0, vecA);
    stage_tile(Bs + buf * KC * m34, m34, G + (int64_t)u0 * m3, m3, KC, m34, un, m3, vecB);
    cp_commit();
  };
  const int tiles = (MT / 4) * (m34 / 4);
  const bool act = threadIdx.x < tiles;
  const int kq = (threadIdx.x % (MT / 4)) * 4, cq = (threadIdx.x / (MT / 4)) * 4;
  T acc[4][4];
  zero4x4(acc);
  if (nchunks > 0) issue(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1, (c + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (act)
      tile4x4(As + (c & 1) * KC * MT, MT, Bs + (c & 1) * KC * m34, m34,
              min(KC, ue - ub - c * KC), kq, cq, acc);
    __syncthreads();
  }
  if (act) {
    T* o = part + (int64_t)blockIdx.y * N3 * m3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + kq + i;
      if (k >= N3) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (cq + j < m3) o[(int64_t)k * m3 + cq + j] = acc[i][j];
    }
  }
}

// tail3: Num3 = sum of splits; MU on F3 rows; BF16 operand of pass 1.
template <typename T>
__global__ void __launch_bounds__(kThreads) tail3_kernel(UpdArgs<T> a, const T* __restrict__ part,
                                                         int splits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int MV = a.mv, S = a.rows_per_block;
  T* hs = sm;             // MV x MV
  T* fo = hs + MV * MV;   // S x MV
  const int64_t r0 = (int64_t)blockIdx.x * S;
  for (int e = threadIdx.x; e < MV * MV; e += blockDim.x) hs[e] = a.H[e];
  for (int e = threadIdx.x; e < S * MV; e += blockDim.x) {
    const int64_t r = r0 + e / MV;
    fo[e] = r < a.nrows ? a.F[r * MV + e % MV] : T(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < S * MV; e += blockDim.x) {
    const int rr = e / MV, v = e % MV;
    const int64_t r = r0 + rr;
    if (r >= a.nrows) continue;
    T num = T(0);
    for (int s = 0; s < splits; ++s) num += part[((int64_t)s * a.nrows + r) * MV + v];
    T den = T(0);
    for (int w = 0; w < MV; ++w) den = fma(fo[rr * MV + w], hs[w * MV + v], den);
    const T nv = mu_step(fo[e], num, den, (T)a.eps);
    a.F[r * MV + v] = nv;
    write_operand(a, r, v, nv);
  }
}

// ---------------------------------------------------------------------------
// core_m: part[s][u][c] = sum_{k in split s} Y3[u, k] F3[k, c]; block (u tile, split).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) core_m_kernel(const T* __restrict__ Y3,
                                                          const T* __restrict__ F3, int UC,
                                                          int N3, int m3, int k_per_split,
                                                          T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int MT = 64, LDA = MT + 4;
  const int m34 = r4(m3);
  T* As = sm;                   // 2 x KC x LDA  (A[k][u], transposed from Y3)
  T* Bs = As + 2 * KC * LDA;    // 2 x KC x m34
  const int u0 = blockIdx.x * MT;
  const int kb = blockIdx.y * k_per_split, ke = min(N3, kb + k_per_split);
  const int nchunks = (ke - kb + KC - 1) / KC;
  const bool vecB = aligned16(F3, m3, sizeof(T));
  auto issue = [&](int c, int buf) {
    const int kc0 = kb + c * KC;
    T* A = As + buf * KC * LDA;
    // A[k][u] = Y3[u0 + u, kc0 + k]: consecutive threads take consecutive k of one row.
    for (int e = threadIdx.x; e < KC * MT; e += blockDim.x) {
      const int uu = e >> 5, kk = e & (KC - 1);
      const bool ok = (u0 + uu < UC) && (kc0 + kk < ke);
      cp_elem(A + kk * LDA + uu, ok ? Y3 + (int64_t)(u0 + uu) * N3 + kc0 + kk : Y3, ok);
    }
    stage_tile(Bs + buf * KC * m34, m34, F3 + (int64_t)kc0 * m3, m3, KC, m34,
               min(KC, ke - kc0), m3, vecB);
    cp_commit();
  };
  const int tiles = (MT / 4) * (m34 / 4);
  const bool act = threadIdx.x < tiles;
  const int uq = (threadIdx.x % (MT / 4)) * 4, cq = (threadIdx.x / (MT / 4)) * 4;
  T acc[4][4];
  zero4x4(acc);
  if (nchunks > 0) issue(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1, (c + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (act)
      tile4x4(As + (c & 1) * KC * LDA, LDA, Bs + (c & 1) * KC * m34, m34,
              min(KC, ke - kb - c * KC), uq, cq, acc);
    __syncthreads();
  }
  if (act) {
    T* o = part + (int64_t)blockIdx.y * UC * m3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = u0 + uq + i;
      if (u >= UC) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (cq + j < m3) o[(int64_t)u * m3 + cq + j] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// core_a: one block per mode-1 index a (no block depends on another):
//   S3 = F3^T F3;  M[a] = sum of the k splits;  D[a] = W3[a] x_3 S3;
//   G[a] <- MU(G[a], M[a], D[a]);  W1[a] = S2 G[a] S3
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) core_a_kernel(CoreArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int m1 = a.m1, m2 = a.m2, m3 = a.m3;
  const int bc = m2 * m3;
  T* s2 = sm;                   // m2 x m2
  T* s3 = s2 + al4(m2 * m2);    // m3 x m3
  T* ga = s3 + al4(m3 * m3);    // bc: G[a] (updated)
  T* wa = ga + al4(bc);         // bc: W3[a], then scratch
  T* stage = wa + al4(bc);      // Gram staging
  const int aa = blockIdx.x;
  const int64_t off = (int64_t)aa * bc;
  for (int e = threadIdx.x; e < m2 * m2; e += blockDim.x) s2[e] = a.S2[e];
  for (int e = threadIdx.x; e < bc; e += blockDim.x) wa[e] = a.W3[off + e];
  gram_block(a.F3, a.n3, m3, s3, stage);  // ends with a barrier
  if (aa == 0)
    for (int e = threadIdx.x; e < m3 * m3; e += blockDim.x) a.S3_out[e] = s3[e];
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {
    const int b = e / m3, c = e % m3;
    T d = T(0);
    for (int w = 0; w < m3; ++w) d = fma(wa[b * m3 + w], s3[w * m3 + c], d);
    T mv = T(0);
    for (int s = 0; s < a.M_splits; ++s) mv += a.M[(int64_t)s * m1 * bc + off + e];
    const T gv = mu_step(a.G[off + e], mv, d, (T)a.eps);
    ga[e] = gv;
    a.G[off + e] = gv;
    a.G2[((int64_t)b * m1 + aa) * m3 + c] = gv;  // G permuted to (m2, m1, m3)
    a.G3[((int64_t)c * m1 + aa) * m2 + b] = gv;  // G permuted to (m3, m1, m2)
    a.Mout[off + e] = mv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {  // scratch = S2 G[a]
    const int b = e / m3, c = e % m3;
    T s = T(0);
    for (int w = 0; w < m2; ++w) s = fma(s2[b * m2 + w], ga[w * m3 + c], s);
    wa[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bc; e += blockDim.x) {  // W1[a] = scratch S3
    const int b = e / m3, c = e % m3;
    T s = T(0);
    for (int w = 0; w < m3; ++w) s = fma(wa[b * m3 + w], s3[w * m3 + c], s);
    a.W1[off + e] = s;
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  __shared__ int last;
  const int m1 = a.m1, m2 = a.m2, m3 = a.m3;
  const int bc = m2 * m3;
  T* wa = sm;  // bc: W1[a]
  const int aa = blockIdx.x;
  const int64_t off = (int64_t)aa * bc;
  for (int e = threadIdx.x; e < bc; e += blockDim.x) wa[e] = a.W1[off + e];
  __syncthreads();
  double mg = 0.0;
  for (int e = threadIdx.x; e < bc; e += blockDim.x)
    mg += (double)a.Mout[off + e] * (double)a.G[off + e];
  mg = block_sum(mg, red);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < m1; q += kThreads / 32) {
    const T s = warp_dot(wa, a.G + (int64_t)q * bc, bc, lane);
    if (lane == 0) a.H1[aa * m1 + q] = s;
  }
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
    if (r2 < 0.0) r2 = 0.0;
    const int t = *a.counter;
    a.trace[(int64_t)t * a.trace_stride] = sqrt(r2 / xx);
    *a.counter = t + 1;
    *a.done = 0;  // ready for the next sweep
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

// S = F^T F for the prologue (one block).
template <typename T>
__global__ void __launch_bounds__(kThreads) gram_kernel(const T* __restrict__ F, int64_t N, int m,
                                                        T* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  gram_block(F, N, m, sm, sm + al4(m * m));
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) S[e] = sm[e];
}

template <typename T>
size_t gram_stage_elems(int m) {
  const int mq = r4(m) / 4, tiles = mq * mq;
  const int groups = kThreads / tiles > 1 ? kThreads / tiles : 1;
  return al4((size_t)gram_rows(m, (int)sizeof(T)) * r4(m)) + (size_t)groups * m * m;
}

int split_count(int64_t blocks, int64_t len, int chunk) {
  const int64_t target = 2LL * device_sm_count();
  int64_t s = (target + blocks - 1) / blocks;
  const int64_t max_s = (len + chunk - 1) / chunk;
  if (s > max_s) s = max_s;
  return (int)(s < 1 ? 1 : s);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <typename T>
int upd_rows_per_block(int mu, int mc, int64_t nrows) {
  const int tiles = (r4(mu) / 4) * (r4(mc) / 4);
  int s = kThreads / tiles;
  if (s < 1) s = 1;
  // Keep about two blocks per SM in flight.
  const int64_t want = (nrows + 2LL * device_sm_count() - 1) / (2LL * device_sm_count());
  if (s > want) s = (int)(want < 1 ? 1 : want);
  return s;
}

template <typename T>
int launch_upd12(const UpdArgs<T>& a, cudaStream_t s) {
  const int tiles = (r4(a.mu) / 4) * (r4(a.mc) / 4);
  if (tiles * a.rows_per_block > kThreads) return NNC_ERR_UNSUPPORTED;
  const int S = a.rows_per_block;
  const size_t smem = sizeof(T) * ((size_t)2 * KC * r4(a.mu) + (size_t)2 * S * KC * r4(a.mc) +
                                   (size_t)S * a.mu * a.mc + (size_t)S * a.mv +
                                   (size_t)a.mv * a.mv + (size_t)S * a.mv);
  NNC_CUDA_TRY(cudaFuncSetAttribute(upd12_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  upd12_kernel<T><<<(unsigned)ceil_div(a.nrows, S), kThreads, smem, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_hmat(const HArgs<T>& a, cudaStream_t s) {
  const size_t g = gram_stage_elems<T>(a.mu) > gram_stage_elems<T>(a.mv) ? gram_stage_elems<T>(a.mu)
                                                                          : gram_stage_elems<T>(a.mv);
  const size_t smem = sizeof(T) * (al4((size_t)a.mu * a.mu) + al4((size_t)a.mv * a.mv) +
                                   3 * al4((size_t)a.mu * a.mv) + g);
  NNC_CUDA_TRY(cudaFuncSetAttribute(hmat_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  hmat_kernel<T><<<a.mp, kThreads, smem, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_y3(const T* P1, const T* F2, int m1, int N2, int N3, int m2, T* Y3, cudaStream_t s) {
  if ((64 / 4) * (r4(m2) / 4) > kThreads) return NNC_ERR_UNSUPPORTED;
  const size_t smem = sizeof(T) * ((size_t)2 * KC * 64 + (size_t)2 * KC * r4(m2));
  NNC_CUDA_TRY(cudaFuncSetAttribute(y3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  dim3 grid((unsigned)ceil_div(N3, 64), (unsigned)m1);
  y3_kernel<T><<<grid, kThreads, smem, s>>>(P1, F2, N2, N3, m2, Y3);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int num3_splits(int UC, int N3) {
  return split_count(ceil_div(N3, 64), UC, KC);
}

template <typename T>
int launch_mode3(const UpdArgs<T>& a, T* part, int splits, cudaStream_t s) {
  const int UC = a.mu, N3 = (int)a.nrows, m3 = a.mv;
  if ((64 / 4) * (r4(m3) / 4) > kThreads) return NNC_ERR_UNSUPPORTED;
  int per = (int)ceil_div(UC, splits);
  per = (int)(ceil_div(per, KC) * KC);
  const int used = (int)ceil_div(UC, per);
  const size_t smem = sizeof(T) * ((size_t)2 * KC * 64 + (size_t)2 * KC * r4(m3));
  NNC_CUDA_TRY(cudaFuncSetAttribute(num3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  dim3 grid((unsigned)ceil_div(N3, 64), (unsigned)used);
  num3_kernel<T><<<grid, kThreads, smem, s>>>(a.P, a.G, UC, N3, m3, per, part);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  const int S = 8;
  UpdArgs<T> t = a;
  t.rows_per_block = S;
  const size_t smem2 = sizeof(T) * ((size_t)m3 * m3 + (size_t)S * m3);
  NNC_CUDA_TRY(cudaFuncSetAttribute(tail3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem2));
  tail3_kernel<T><<<(unsigned)ceil_div(N3, S), kThreads, smem2, s>>>(t, part, used);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int core_m_splits(int UC, int N3) {
  return split_count(ceil_div(UC, 64), N3, KC);
}

template <typename T>
int launch_core_m(const T* Y3, const T* F3, int UC, int N3, int m3, T* part, int splits,
                  int* used_splits, cudaStream_t s) {
  if ((64 / 4) * (r4(m3) / 4) > kThreads) return NNC_ERR_UNSUPPORTED;
  int per = (int)ceil_div(N3, splits);
  per = (int)(ceil_div(per, KC) * KC);
  const int used = (int)ceil_div(N3, per);
  const size_t smem = sizeof(T) * ((size_t)2 * KC * 68 + (size_t)2 * KC * r4(m3));
  NNC_CUDA_TRY(cudaFuncSetAttribute(core_m_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  dim3 grid((unsigned)ceil_div(UC, 64), (unsigned)used);
  core_m_kernel<T><<<grid, kThreads, smem, s>>>(Y3, F3, UC, N3, m3, per, part);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  *used_splits = used;
  return NNC_OK;
}

template <typename T>
int launch_core(const CoreArgs<T>& a, cudaStream_t s) {
  const size_t bc = (size_t)a.m2 * a.m3;
  const size_t smem_a = sizeof(T) * (al4((size_t)a.m2 * a.m2) + al4((size_t)a.m3 * a.m3) +
                                     2 * al4(bc) + gram_stage_elems<T>(a.m3));
  NNC_CUDA_TRY(cudaFuncSetAttribute(core_a_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_a));
  core_a_kernel<T><<<a.m1, kThreads, smem_a, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  const size_t smem_b = sizeof(T) * al4(bc);
  NNC_CUDA_TRY(cudaFuncSetAttribute(core_b_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_b));
  core_b_kernel<T><<<a.m1, kThreads, smem_b, s>>>(a);
  note_launch(s);
  NNC_CUDA_TRY(cudaGetLastError());
  return NNC_OK;
}

template <typename T>
int launch_gram(const T* F, int64_t N, int m, T* S, cudaStream_t s) {
  const size_t smem = sizeof(T) * (al4((size_t)m * m) + gram_stage_elems<T>(m));
  NNC_CUDA_TRY(cudaFuncSetAttribute(gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
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
  template int upd_rows_per_block<T>(int, int, int64_t);                                    \
  template int launch_upd12<T>(const UpdArgs<T>&, cudaStream_t);                            \
  template int launch_hmat<T>(const HArgs<T>&, cudaStream_t);                               \
  template int launch_y3<T>(const T*, const T*, int, int, int, int, T*, cudaStream_t);      \
  template int num3_splits<T>(int, int);                                                    \
  template int launch_mode3<T>(const UpdArgs<T>&, T*, int, cudaStream_t);                   \
  template int core_m_splits<T>(int, int);                                                  \
  template int launch_core_m<T>(const T*, const T*, int, int, int, T*, int, int*,           \
                                cudaStream_t);                                              \
  template int launch_core<T>(const CoreArgs<T>&, cudaStream_t);                            \
  template int launch_gram<T>(const T*, int64_t, int, T*, cudaStream_t);                    \
  template int launch_permute_core<T>(const T*, int, int, int, T*, T*, cudaStream_t);
NNC_SWEEP_INST(float)
NNC_SWEEP_INST(double)
#undef NNC_SWEEP_INST

}  // namespace nnc
