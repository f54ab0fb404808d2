// A 32 x 32 FP32 tile Z += A^T B on the tensor cores (mma.sync m16n8k8, TF32
// operands, FP32 accumulation), from operands staged with rows of 32 FP32
// entries in the 128-byte swizzle (16-byte chunk v of row k at chunk
// v ^ (k % 8)). Used by the factor updates (sweep.cu) and by the fused tile
// contraction of the pass epilogue (tc_ttm.cu).
//
// A warp holds the whole tile: acc[i][j][q] is entry (s, c) of Z with
//   s = 4 g + 2 i + q / 2,   c = 8 t + 4 (q % 2) + j,   (g, t) = (lane / 4, lane % 4).
// The MMA's labels are permuted so that thread (g, t) reads its fragments with
// one 16-byte load per operand row: logical row rho of M-tile i is entry
// 4 (rho % 8) + 2 i + rho / 8 of A's row, logical column n of N-tile j entry
// 4 n + j of B's row, and within each 8-row step the MMA's k = t is row 2t and
// k = t + 4 row 2t + 1 (the same for both operands). With the swizzle, the
// eight lanes of a quarter warp then load from eight distinct 16-byte bank
// groups.
#pragma once

#include <cstdint>

namespace nnc {
namespace mma32 {

// x rounded to TF32 (10 stored mantissa bits), to nearest with ties away from
// zero: half of the dropped 13-bit field is added to the sign-magnitude bits
// and the field cleared (a carry moves into the exponent). Finite inputs stay
// finite below (2 - 2^-11) 2^127; infinities and NaNs stay what they are.
__device__ __forceinline__ uint32_t tf32_rn(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// d += a b for one m16n8k8 tile.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// This thread's two row offsets (in floats) within an 8-row step.
__device__ __forceinline__ int frag_off(int lane, int h) {
  const int g = lane >> 2, k = 2 * (lane & 3) + h;
  return k * 32 + 4 * (g ^ k);
}

__device__ __forceinline__ void zero(float (&acc)[2][4][4]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
}

// One 8-row step from A rows at `a` and B rows at `b` (the step's first row;
// o0, o1 from frag_off). SPLIT = 1: operands rounded to TF32. SPLIT = 3: every
// operand x split into x_hi = tf32(x) and x_lo = tf32(x - x_hi), and
// x_lo y_hi + x_hi y_lo + x_hi y_hi accumulated (the dropped x_lo y_lo is below
// FP32 rounding): FP32-accurate.
template <int SPLIT>
__device__ __forceinline__ void step(float (&acc)[2][4][4], const float* a, const float* b,
                                     int o0, int o1) {
  float xa[2][4], xb[2][4];
  {
    const float4 p = *reinterpret_cast<const float4*>(a + o0);
    const float4 q = *reinterpret_cast<const float4*>(a + o1);
    const float4 u = *reinterpret_cast<const float4*>(b + o0);
    const float4 v = *reinterpret_cast<const float4*>(b + o1);
    xa[0][0] = p.x; xa[0][1] = p.y; xa[0][2] = p.z; xa[0][3] = p.w;
    xa[1][0] = q.x; xa[1][1] = q.y; xa[1][2] = q.z; xa[1][3] = q.w;
    xb[0][0] = u.x; xb[0][1] = u.y; xb[0][2] = u.z; xb[0][3] = u.w;
    xb[1][0] = v.x; xb[1][1] = v.y; xb[1][2] = v.z; xb[1][3] = v.w;
  }
  uint32_t ah[2][4], bh[4][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) ah[i][e] = tf32_rn(xa[e >> 1][2 * i + (e & 1)]);
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) bh[j][h] = tf32_rn(xb[h][j]);
  if constexpr (SPLIT == 3) {
    uint32_t al[2][4], bl[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        al[i][e] = tf32_rn(xa[e >> 1][2 * i + (e & 1)] - __uint_as_float(ah[i][e]));
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) bl[j][h] = tf32_rn(xb[h][j] - __uint_as_float(bh[j][h]));
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        mma_tf32(acc[i][j], al[i], bh[j][0], bh[j][1]);
        mma_tf32(acc[i][j], ah[i], bl[j][0], bl[j][1]);
      }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) mma_tf32(acc[i][j], ah[i], bh[j][0], bh[j][1]);
}

// Entry (s, c) of the tile in a 32 x 32 shared-memory buffer whose rows have
// their 4-entry groups permuted so that the per-thread stores of `store`
// fall on 32 distinct banks.
__device__ __forceinline__ int tile_index(int s, int c) { return s * 32 + (c ^ ((s >> 2) & 7)); }

__device__ __forceinline__ void store(float* z, const float (&acc)[2][4][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        z[tile_index(4 * g + 2 * i + (q >> 1), 8 * t + 4 * (q & 1) + j)] = acc[i][j][q];
}

}  // namespace mma32
}  // namespace nnc
