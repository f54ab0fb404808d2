// SIMT mode products (n-mode multiplication, Appendix A) used by the FP32 and
// FP64 paths: the two passes over X of every sweep and all the small
// contractions around them.
//
// A tensor is viewed as (L, J, C) with J the contracted mode:
//   out[l, q, c] = sum_j Fm[j, q] * Y[l, j, c]
// Two kernels cover the two memory patterns:
//   * ttm_rows (C == 1): J is the contiguous axis (e.g. X x_3 F^(3)T). A block
//     stages a BM x 32 tile of Y and a 32 x QP slice of Fm in shared memory;
//     each thread keeps TR rows x QP outputs in registers.
//   * ttm_cols (C > 1): J is strided (e.g. X x_1 F^(1)T). Each thread owns TC
//     flattened (l, c) columns, streams them along j with coalesced loads and
//     keeps QP outputs per column in registers; Fm rows are broadcast from
//     shared memory.
//   * ttm_cols_pipe (C > 1, rows of C 16-byte aligned): the same register
//     tiling, with the block's 256 TC flattened columns staged through a
//     3-deep cp.async ring of 16 rows j, so that two chunks are in flight
//     while the third is consumed.
//   * ttm_cols_tc (float, C % 4 == 0, Q <= 32): the column product as a GEMM on
//     the tensor cores (TF32x3 on mma.sync, FP32-accurate), for the mode
//     products of the compressed tensors in the tensor-core paths.
// All accumulate in T and, when one pass would not fill the GPU, split J
// across blocks; partial sums are then added in split order (deterministic).
#include <type_traits>

#include "kernels.cuh"
#include "mma32.cuh"

namespace nnc {
namespace {

constexpr int kRowsThreads = 128;
// K-chunk of ttm_rows: 32 for float, 16 for double (static shared memory < 48 KB).
template <typename T>
__host__ __device__ constexpr int rows_bk() { return sizeof(T) == 4 ? 32 : 16; }
constexpr int kColsThreads = 256;
constexpr int kColsBJ = 32;

template <typename T, int QP, int TR>
__global__ void __launch_bounds__(kRowsThreads)
ttm_rows_kernel(const T* __restrict__ Y, int64_t R, int K, int k_per_split,
                const T* __restrict__ Fm, int64_t fs_k, int64_t fs_q, int Q,
                T* __restrict__ out) {
  constexpr int BM = kRowsThreads * TR;
  constexpr int BK = rows_bk<T>();
  __shared__ T Xs[BM][BK + 1];
  __shared__ __align__(16) T Fs[BK][QP];

  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * BM;
  const int kbeg = blockIdx.y * k_per_split;
  const int kend = min(K, kbeg + k_per_split);

  T acc[TR][QP];
#pragma unroll
  for (int t = 0; t < TR; ++t)
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[t][q] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BM * BK; e += kRowsThreads) {
      const int rr = e / BK, kk = e % BK;
      const int64_t r = r0 + rr;
      const int k = k0 + kk;
      Xs[rr][kk] = (r < R && k < kend) ? Y[r * K + k] : T(0);
    }
    for (int e = tid; e < BK * QP; e += kRowsThreads) {
      const int kk = e / QP, q = e % QP;
      const int k = k0 + kk;
      Fs[kk][q] = (q < Q && k < kend) ? Fm[k * fs_k + q * fs_q] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      T x[TR];
#pragma unroll
      for (int t = 0; t < TR; ++t) x[t] = Xs[tid + t * kRowsThreads][kk];
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const T f = Fs[kk][q];
#pragma unroll
        for (int t = 0; t < TR; ++t) acc[t][q] = fma(x[t], f, acc[t][q]);
      }
    }
    __syncthreads();
  }

  T* o = out + (int64_t)blockIdx.y * R * Q;
#pragma unroll
  for (int t = 0; t < TR; ++t) {
    const int64_t r = r0 + tid + t * kRowsThreads;
    if (r < R) {
#pragma unroll
      for (int q = 0; q < QP; ++q)
        if (q < Q) o[r * Q + q] = acc[t][q];
    }
  }
}

template <typename T, int QP, int TC>
__global__ void __launch_bounds__(kColsThreads)
ttm_cols_kernel(const T* __restrict__ Y, int64_t L, int J, int64_t C, int j_per_split,
                const T* __restrict__ Fm, int64_t fs_j, int64_t fs_q, int Q,
                T* __restrict__ out) {
  constexpr int BJ = kColsBJ;
  __shared__ __align__(16) T Fs[BJ][QP];

  const int64_t ncols = L * C;
  const int64_t base = (int64_t)blockIdx.x * (kColsThreads * TC) + threadIdx.x;
  const int jbeg = blockIdx.y * j_per_split;
  const int jend = min(J, jbeg + j_per_split);

  const T* y[TC];
  int64_t col_l[TC], col_c[TC];
  bool active[TC];
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int64_t g = base + (int64_t)t * kColsThreads;
    active[t] = g < ncols;
    const int64_t gg = active[t] ? g : 0;
    col_l[t] = gg / C;
    col_c[t] = gg % C;
    y[t] = Y + col_l[t] * (int64_t)J * C + col_c[t];
  }

  T acc[TC][QP];
#pragma unroll
  for (int t = 0; t < TC; ++t)
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[t][q] = T(0);

  for (int j0 = jbeg; j0 < jend; j0 += BJ) {
    for (int e = threadIdx.x; e < BJ * QP; e += kColsThreads) {
      const int jj = e / QP, q = e % QP;
      const int j = j0 + jj;
      Fs[jj][q] = (q < Q && j < jend) ? Fm[j * fs_j + q * fs_q] : T(0);
    }
    __syncthreads();
    const int jn = min(BJ, jend - j0);
#pragma unroll 4
    for (int jj = 0; jj < jn; ++jj) {
      T v[TC];
#pragma unroll
      for (int t = 0; t < TC; ++t) v[t] = active[t] ? y[t][(int64_t)(j0 + jj) * C] : T(0);
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const T f = Fs[jj][q];
#pragma unroll
        for (int t = 0; t < TC; ++t) acc[t][q] = fma(f, v[t], acc[t][q]);
      }
    }
    __syncthreads();
  }

  T* o = out + (int64_t)blockIdx.y * L * Q * C;
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    if (!active[t]) continue;
    T* ot = o + col_l[t] * Q * C + col_c[t];
#pragma unroll
    for (int q = 0; q < QP; ++q)
      if (q < Q) ot[(int64_t)q * C] = acc[t][q];
  }
}

constexpr int kPipeBJ = 16;
constexpr int kPipeStages = 3;

template <typename T, int QP, int TC>
constexpr size_t pipe_smem_bytes() {
  return (size_t)kPipeStages * kPipeBJ * (kColsThreads * TC + QP) * sizeof(T);
}

// Flattened columns (l, c) col0 .. col0 + BC - 1 (BC = 256 TC, col0 =
// blockIdx.x BC), rows j of split blockIdx.y. Each 16-byte copy stays in one
// row (l, j) because C % V == 0. Rows and columns past the ends are staged as
// zeros (Fm rows too), so every chunk runs all kPipeBJ rows.
template <typename T, int QP, int TC>
__global__ void __launch_bounds__(kColsThreads, QP * TC * sizeof(T) < 256 ? 2 : 1)
ttm_cols_pipe_kernel(const T* __restrict__ Y, int64_t L, int J, int64_t C, int j_per_split, const T* __restrict__ Fm, int64_t fs_j, int64_t fs_q, int Q,
                     T* __restrict__ out) {
  constexpr int BC = kColsThreads * TC;
  constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte copy
  constexpr int CPR = BC / V;             // copies per staged row
  static_assert(QP % V == 0, "QP must be a whole number of 16-byte vectors");
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ys = reinterpret_cast<T*>(smem_raw);      // [stage][kPipeBJ][BC]
  T* Fs = Ys + kPipeStages * kPipeBJ * BC;     // [stage][kPipeBJ][QP]
  const int tid = threadIdx.x;
  const int64_t ncols = L * C;
  const int64_t col0 = (int64_t)blockIdx.x * BC;
  const int jbeg = blockIdx.y * j_per_split;
  const int jend = min(J, jbeg + j_per_split);
  const int nchunks = (jend - jbeg + kPipeBJ - 1) / kPipeBJ;

  // This thread's copies: vector v of the rows jr, jr + RP, ... of a chunk.
  constexpr int RP = kColsThreads / CPR;
  static_assert(kColsThreads % CPR == 0 && kPipeBJ % RP == 0, "copy layout");
  const int v = tid % CPR, jr = tid / CPR;
  const int64_t vcol = col0 + (int64_t)v * V;
  const bool cok = vcol < ncols;
  const int64_t vl = cok ? vcol / C : 0;
  const T* ysrc = Y + vl * (int64_t)J * C + (cok ? vcol - vl * C : 0);
  auto issue = [&](int chunk) {
    const int slot = chunk % kPipeStages;
    const int j0 = jbeg + chunk * kPipeBJ;
    T* ys = Ys + slot * kPipeBJ * BC + v * V;
#pragma unroll
    for (int jj = jr; jj < kPipeBJ; jj += RP) {
      const int j = j0 + jj;
      const bool ok = cok && j < jend;
      cp_vec(ys + jj * BC, ok ? ysrc + (int64_t)j * C : Y, ok ? V : 0);
    }
    // The Fm rows of the chunk go the same way (element copies), so that no
    // thread waits for them before the chunk it is about to consume.
    T* fs = Fs + slot * kPipeBJ * QP;
    for (int e = tid; e < kPipeBJ * QP; e += kColsThreads) {
      const int jj = e / QP, q = e % QP;
      const int j = j0 + jj;
      const bool ok = q < Q && j < jend;
      cp_elem(fs + e, ok ? Fm + (j * fs_j + q * fs_q) : Fm, ok);
    }
  };

  T acc[TC][QP];
#pragma unroll
  for (int t = 0; t < TC; ++t)
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[t][q] = T(0);

#pragma unroll
  for (int p = 0; p < kPipeStages - 1; ++p) {
    if (p < nchunks) issue(p);
    cp_commit();
  }
  for (int it = 0; it < nchunks; ++it) {
    if (it + kPipeStages - 1 < nchunks) issue(it + kPipeStages - 1);
    cp_commit();
    cp_wait<kPipeStages - 1>();
    __syncthreads();
    const int slot = it % kPipeStages;
    const T* ys = Ys + slot * kPipeBJ * BC;
    const T* fs = Fs + slot * kPipeBJ * QP;
#pragma unroll 4
    for (int jj = 0; jj < kPipeBJ; ++jj) {
      T v[TC];
#pragma unroll
      for (int t = 0; t < TC; ++t) v[t] = ys[jj * BC + tid + t * kColsThreads];
      const Vec* fr = reinterpret_cast<const Vec*>(fs + jj * QP);
#pragma unroll
      for (int g = 0; g < QP / V; ++g) {
        const Vec f4 = fr[g];
        T f[V];
        if constexpr (sizeof(T) == 4) {
          f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
        } else {
          f[0] = f4.x; f[1] = f4.y;
        }
#pragma unroll
        for (int u = 0; u < V; ++u)
#pragma unroll
          for (int t = 0; t < TC; ++t) acc[t][g * V + u] = fma(f[u], v[t], acc[t][g * V + u]);
      }
    }
    __syncthreads();
  }

  T* o = out + (int64_t)blockIdx.y * L * Q * C;
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int64_t col = col0 + tid + t * kColsThreads;
    if (col >= ncols) continue;
    const int64_t l = col / C;
    T* ot = o + l * Q * C + (col - l * C);
#pragma unroll
    for (int q = 0; q < QP; ++q)
      if (q < Q) ot[(int64_t)q * C] = acc[t][q];
  }
}

// Tensor-core column mode product (float, C % 4 == 0, Q <= 32): per block the
// GEMM D (kTcCols columns (l, c) x QP) = A (columns x rows j) B (rows j x QP),
// A the staged rows of Y (a column is an MMA row, j the MMA k), B the rows of
// Fm, on mma.sync m16n8k8 with TF32x3 operands (x = x_hi + x_lo, the three
// products lo*hi, hi*lo, hi*hi; the dropped lo*lo is below FP32 rounding) and
// FP32 accumulation. Each chunk of kTcBJ rows is summed in a fresh fragment
// and then added to the running sum with round-to-nearest, so the tensor
// core's truncating accumulation only ever acts on one chunk's sum. The rows
// are staged as in ttm_cols_pipe (a cp.async ring; rows and columns past the
// ends are zeros). Warp w owns columns 32 w .. 32 w + 31 (two M-tiles).
constexpr int kTcCols = 256;
constexpr int kTcBJ = 16;
constexpr int kTcStages = 4;
constexpr int kTcYS = kTcCols + 8;  // row stride: the A fragments hit 32 distinct banks

template <int QP>
__host__ __device__ constexpr int tc_fs() { return QP == 24 ? 24 : QP + 8; }
template <int QP>
constexpr size_t tc_smem_bytes() {
  return (size_t)kTcStages * kTcBJ * (kTcYS + tc_fs<QP>()) * sizeof(float);
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = mma32::tf32_rn(x);
  lo = mma32::tf32_rn(x - __uint_as_float(hi));
}

template <int QP>
__global__ void __launch_bounds__(kColsThreads, 2)
ttm_cols_tc_kernel(const float* __restrict__ Y, int64_t L, int J, int64_t C, int j_per_split,
                   const float* __restrict__ Fm, int64_t fs_j, int64_t fs_q, int Q,
                   float* __restrict__ out) {
  static_assert(kColsThreads == 256 && kTcCols == 256, "eight warps of 32 columns");
  constexpr int NT = QP / 8;
  constexpr int FS = tc_fs<QP>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);  // [stage][kTcBJ][kTcYS]
  float* Fs = Ys + kTcStages * kTcBJ * kTcYS;       // [stage][kTcBJ][FS]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t ncols = L * C;
  const int64_t col0 = (int64_t)blockIdx.x * kTcCols;
  const int jbeg = blockIdx.y * j_per_split;
  const int jend = min(J, jbeg + j_per_split);
  const int nchunks = (jend - jbeg + kTcBJ - 1) / kTcBJ;

  // This thread's copies: 16-byte vector v of rows jr, jr + 4, ... of a chunk
  // (a vector never crosses a row (l, j) because C % 4 == 0).
  const int v = tid & 63, jr = tid >> 6;
  const int64_t vcol = col0 + (int64_t)v * 4;
  const bool cok = vcol < ncols;
  const int64_t vl = cok ? vcol / C : 0;
  const float* ysrc = Y + vl * (int64_t)J * C + (cok ? vcol - vl * C : 0);
  auto issue = [&](int chunk) {
    const int slot = chunk % kTcStages;
    const int j0 = jbeg + chunk * kTcBJ;
    float* ys = Ys + slot * kTcBJ * kTcYS + v * 4;
#pragma unroll
    for (int jj = jr; jj < kTcBJ; jj += 4) {
      const int j = j0 + jj;
      const bool ok = cok && j < jend;
      cp_vec(ys + jj * kTcYS, ok ? ysrc + (int64_t)j * C : Y, ok ? 4 : 0);
    }
    float* fs = Fs + slot * kTcBJ * FS;
    for (int e = tid; e < kTcBJ * QP; e += kColsThreads) {
      const int jj = e / QP, q = e % QP;
      const int j = j0 + jj;
      const bool ok = q < Q && j < jend;
      cp_elem(fs + jj * FS + q, ok ? Fm + (j * fs_j + q * fs_q) : Fm, ok);
    }
  };

  float acc[2][NT][4], part[2][NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][n][e] = part[i][n][e] = 0.f;

#pragma unroll
  for (int p = 0; p < kTcStages - 1; ++p) {
    if (p < nchunks) issue(p);
    cp_commit();
  }
  for (int it = 0; it < nchunks; ++it) {
    if (it + kTcStages - 1 < nchunks) issue(it + kTcStages - 1);
    cp_commit();
    cp_wait<kTcStages - 1>();
    __syncthreads();
    const int slot = it % kTcStages;
    const float* ys = Ys + slot * kTcBJ * kTcYS + warp * 32 + g;
    const float* fs = Fs + slot * kTcBJ * FS + g;
#pragma unroll
    for (int ks = 0; ks < kTcBJ / 8; ++ks) {
      const float* y0 = ys + (ks * 8 + t) * kTcYS;
      const float* y1 = y0 + 4 * kTcYS;
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        split_tf32(y0[16 * i], ah[i][0], al[i][0]);
        split_tf32(y0[16 * i + 8], ah[i][1], al[i][1]);
        split_tf32(y1[16 * i], ah[i][2], al[i][2]);
        split_tf32(y1[16 * i + 8], ah[i][3], al[i][3]);
      }
      const float* f0 = fs + (ks * 8 + t) * FS;
      const float* f1 = f0 + 4 * FS;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(f0[8 * n], bh0, bl0);
        split_tf32(f1[8 * n], bh1, bl1);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma32::mma_tf32(part[i][n], al[i], bh0, bh1);
          mma32::mma_tf32(part[i][n], ah[i], bl0, bl1);
          mma32::mma_tf32(part[i][n], ah[i], bh0, bh1);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc[i][n][e] += part[i][n][e];
          part[i][n][e] = 0.f;
        }
  }

  // D fragment: entry e of tile (i, n) is column 32 warp + 16 i + g + 8 (e / 2),
  // q = 8 n + 2 t + e % 2.
  float* o = out + (int64_t)blockIdx.y * L * Q * C;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t col = col0 + warp * 32 + 16 * i + g + 8 * h;
      if (col >= ncols) continue;
      const int64_t l = col / C;
      float* ot = o + l * Q * C + (col - l * C);
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int q = 8 * n + 2 * t + u;
          if (q < Q) ot[(int64_t)q * C] = acc[i][n][2 * h + u];
        }
    }
}

template <typename T>
__global__ void reduce_splits_kernel(const T* __restrict__ part, int splits, int64_t n,
                                     T* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // Loads in groups of 8 (all in flight together), added in split order.
    T s = part[i];
    int p = 1;
    for (; p + 8 <= splits; p += 8) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = part[(int64_t)(p + u) * n + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; p < splits; ++p) s += part[(int64_t)p * n + i];
    out[i] = s;
  }
}

// Number of J-splits so that about two blocks per SM are in flight, bounded by
// the scratch capacity and by one 32-wide chunk of J per split.
int choose_splits(int64_t blocks, int J, int64_t out_elems, size_t split_cap, int chunk,
                  int* per_split) {
  const int64_t target = 2LL * device_sm_count();
  int splits = 1;
  if (blocks < target && J >= 2 * chunk && split_cap > 0) {
    int64_t want = ceil_div(target, blocks);
    int64_t by_j = J / chunk;
    int64_t by_cap = (int64_t)(split_cap / (size_t)out_elems);
    int64_t s = want;
    if (s > by_j) s = by_j;
    if (s > by_cap) s = by_cap;
    if (s > 1) splits = (int)s;
  }
  int per = (int)ceil_div(J, splits);
  per = (int)(ceil_div(per, chunk) * chunk);
  *per_split = per;
  return (int)ceil_div(J, per);
}

template <typename T, int QP>
cudaError_t ttm_dispatch(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                         int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                         cudaStream_t s) {
  const int64_t out_elems = L * Q * C;
  int per = J, splits = 1;
  if (C == 1) {
    constexpr int TR = (sizeof(T) == 4 && QP <= 32) ? 2 : 1;
    constexpr int BM = kRowsThreads * TR;
    const int64_t blocks = ceil_div(L, BM);
    splits = choose_splits(blocks, J, out_elems, split_cap, rows_bk<T>(), &per);
    T* dst = splits > 1 ? split_buf : out;
    dim3 grid((unsigned)blocks, (unsigned)splits);
    ttm_rows_kernel<T, QP, TR><<<grid, kRowsThreads, 0, s>>>(Y, L, J, per, Fm, fs_j, fs_q, Q, dst);
    note_launch(s);
  } else {
    const int64_t ncols = L * C;
    const bool wide = (QP <= 32) && ceil_div(ncols, 2 * kColsThreads) >= 2LL * device_sm_count();
    constexpr int PV = 16 / (int)sizeof(T);
    const bool pipe = C % PV == 0 && reinterpret_cast<uintptr_t>(Y) % 16 == 0;
    if (pipe) {
      // Two columns per thread when the grid still has two blocks per SM.
      constexpr bool two = sizeof(T) == 4 && QP <= 32;
      const bool use2 = two && ceil_div(ncols, 2 * kColsThreads) >= 2LL * device_sm_count();
      const int64_t blocks = ceil_div(ncols, (int64_t)(use2 ? 2 : 1) * kColsThreads);
      if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
      splits = choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
      T* dst = splits > 1 ? split_buf : out;
      dim3 grid((unsigned)blocks, (unsigned)splits);
      if (use2) {
        constexpr int PTC = two ? 2 : 1;
        constexpr size_t smem = pipe_smem_bytes<T, QP, PTC>();
        const cudaError_t e0 =
            raise_smem_limit((const void*)ttm_cols_pipe_kernel<T, QP, PTC>, smem);
        if (e0 != cudaSuccess) return e0;
        ttm_cols_pipe_kernel<T, QP, PTC><<<grid, kColsThreads, smem, s>>>(
            Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
      } else {
        constexpr size_t smem = pipe_smem_bytes<T, QP, 1>();
        const cudaError_t e0 = raise_smem_limit((const void*)ttm_cols_pipe_kernel<T, QP, 1>, smem);
        if (e0 != cudaSuccess) return e0;
        ttm_cols_pipe_kernel<T, QP, 1><<<grid, kColsThreads, smem, s>>>(Y, L, J, C, per, Fm, fs_j,
                                                                         fs_q, Q, dst);
      }
      note_launch(s);
    } else if (wide) {
      const int64_t blocks = ceil_div(ncols, 2 * kColsThreads);
      splits = choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
      T* dst = splits > 1 ? split_buf : out;
      dim3 grid((unsigned)blocks, (unsigned)splits);
      ttm_cols_kernel<T, QP, 2><<<grid, kColsThreads, 0, s>>>(Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
      note_launch(s);
    } else {
      const int64_t blocks = ceil_div(ncols, kColsThreads);
      splits = choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
      T* dst = splits > 1 ? split_buf : out;
      dim3 grid((unsigned)blocks, (unsigned)splits);
      ttm_cols_kernel<T, QP, 1><<<grid, kColsThreads, 0, s>>>(Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
      note_launch(s);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t blocks = ceil_div(out_elems, 256) < 4096 ? ceil_div(out_elems, 256) : 4096;
  reduce_splits_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(split_buf, splits, out_elems, out);
  note_launch(s);
  return cudaGetLastError();
}

template <int QP>
cudaError_t ttm_tc_dispatch(const float* Y, int64_t L, int J, int64_t C, const float* Fm,
                            int64_t fs_j, int64_t fs_q, int Q, float* out, float* split_buf,
                            size_t split_cap, cudaStream_t s) {
  const int64_t ncols = L * C, out_elems = L * Q * C;
  const int64_t blocks = ceil_div(ncols, kTcCols);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  // Two or three blocks fit on an SM, so a grid of at least one block per SM
  // runs in one wave: J is split (with a second launch for the sums) only
  // below that (measured on the 4-way sweep's chains: 0.7 % faster per sweep).
  int per = J;
  const int splits = blocks >= device_sm_count()
                         ? 1
                         : choose_splits(blocks, J, out_elems, split_cap, kColsBJ, &per);
  float* dst = splits > 1 ? split_buf : out;
  constexpr size_t smem = tc_smem_bytes<QP>();
  const cudaError_t e0 = raise_smem_limit((const void*)ttm_cols_tc_kernel<QP>, smem);
  if (e0 != cudaSuccess) return e0;
  dim3 grid((unsigned)blocks, (unsigned)splits);
  ttm_cols_tc_kernel<QP><<<grid, kColsThreads, smem, s>>>(Y, L, J, C, per, Fm, fs_j, fs_q, Q, dst);
  note_launch(s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t rb = ceil_div(out_elems, 256) < 4096 ? ceil_div(out_elems, 256) : 4096;
  reduce_splits_kernel<float><<<(unsigned)rb, 256, 0, s>>>(split_buf, splits, out_elems, out);
  note_launch(s);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_ttm(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                       int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                       cudaStream_t s) {
  if (L <= 0 || J <= 0 || C <= 0 || Q <= 0) return cudaErrorInvalidValue;
  if (Q <= 8) return ttm_dispatch<T, 8>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 16) return ttm_dispatch<T, 16>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 24) return ttm_dispatch<T, 24>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 32) return ttm_dispatch<T, 32>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  if (Q <= 64) return ttm_dispatch<T, 64>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ttm_tc(const T* Y, int64_t L, int J, int64_t C, const T* Fm, int64_t fs_j,
                          int64_t fs_q, int Q, T* out, T* split_buf, size_t split_cap,
                          cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (L > 0 && J > 0 && C > 1 && Q > 0 && Q <= 32 && C % 4 == 0 &&
        reinterpret_cast<uintptr_t>(Y) % 16 == 0) {
      if (Q <= 16)
        return ttm_tc_dispatch<16>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
      if (Q <= 24)
        return ttm_tc_dispatch<24>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
      return ttm_tc_dispatch<32>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
    }
  }
  return launch_ttm<T>(Y, L, J, C, Fm, fs_j, fs_q, Q, out, split_buf, split_cap, s);
}

template <typename T>
cudaError_t launch_reduce_splits(const T* part, int splits, int64_t n, T* out, cudaStream_t s) {
  const int64_t blocks = ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096;
  reduce_splits_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(part, splits, n, out);
  note_launch(s);
  return cudaGetLastError();
}

template cudaError_t launch_reduce_splits<float>(const float*, int, int64_t, float*,
                                                 cudaStream_t);
template cudaError_t launch_reduce_splits<double>(const double*, int, int64_t, double*,
                                                  cudaStream_t);
template cudaError_t launch_ttm_tc<float>(const float*, int64_t, int, int64_t, const float*,
                                          int64_t, int64_t, int, float*, float*, size_t,
                                          cudaStream_t);
template cudaError_t launch_ttm_tc<double>(const double*, int64_t, int, int64_t, const double*,
                                           int64_t, int64_t, int, double*, double*, size_t,
                                           cudaStream_t);
template cudaError_t launch_ttm<float>(const float*, int64_t, int, int64_t, const float*, int64_t,
                                       int64_t, int, float*, float*, size_t, cudaStream_t);
template cudaError_t launch_ttm<double>(const double*, int64_t, int, int64_t, const double*,
                                        int64_t, int64_t, int, double*, double*, size_t,
                                        cudaStream_t);

}  // namespace nnc
