// top_tc.cuh -- the local step's product ch = G rhs (Eq. 18a) on the tensor
// cores, for a warp whose 32 segments share one inverse G = (D K D)^-1.
//
// Segments that share a duration (the interior segments of a trajectory with
// one T, Sec. III-D.1) share G, so a warp's 32 x 3 right-hand sides form one
// product G (8 x 8) * RHS (8 x 96).  It runs as twelve mma.sync m16n8k8 tiles
// (one per axis and eight segments) with TF32 operands.  TF32 keeps 10
// mantissa bits, so both operands are split into a high and a low TF32 part
// and three products are kept (hi*hi + hi*lo + lo*hi, the error of the
// dropped lo*lo term is ~2^-22 relative): the A operand stacks G_hi over
// G_lo in its 16 rows, so two MMAs per tile give G_hi B_hi, G_lo B_hi (rows
// 8-15) and G_hi B_lo, accumulated in FP32.
//
// The operands travel through the warp's rows of a shared-memory scratch of
// 28 floats per segment (stride 28: the fragment loads and the result stores
// are free of bank conflicts): each lane writes its 24 right-hand-side values
// to its row, loads its B fragments from the rows of the tile's segments,
// stores its D fragments into those rows, and reads its 24 coefficients back
// from its own row.
#pragma once

#include <cstdint>

#include "top_math.cuh"

namespace top {

constexpr int kTcRow = 28;  // scratch floats per segment

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// d = A B + c for one m16n8k8 tile (A 16x8 row-major, B 8x8 column-major, TF32)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1, const float (&c)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// The A fragments of [G_hi; G_lo]: lane (g = lane / 4, t = lane % 4) holds
// rows g and g + 8, columns t and t + 4.  Gseg points at this lane's own
// segment column of the packed inverses ([36][S], stride S): every lane of
// the warp holds the shared G.
struct TcA {
  uint32_t hi0, lo0, hi1, lo1;  // G_hi[g][t], G_lo[g][t], G_hi[g][t+4], G_lo[g][t+4]
};

__device__ __forceinline__ TcA tc_a_fragments(const float *Gseg, size_t S, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const float x0 = Gseg[(size_t)gidx(g, t) * S], x1 = Gseg[(size_t)gidx(g, t + 4) * S];
  TcA A;
  A.hi0 = tf32_rna(x0);
  A.lo0 = tf32_rna(x0 - __uint_as_float(A.hi0));
  A.hi1 = tf32_rna(x1);
  A.lo1 = tf32_rna(x1 - __uint_as_float(A.hi1));
  return A;
}

// ch = G rhs for the warp's 32 segments; every lane of the warp calls it.
// scr: the warp's first scratch row (32 rows of kTcRow floats).
__device__ __forceinline__ void apply_g_mma(const TcA &A, const float (&rhs)[AX][NC], float (&ch)[AX][NC],
                                            float *scr, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float *mine = scr + lane * kTcRow;
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) mine[a * NC + k] = rhs[a][k];
  __syncwarp();
  float out[12][2];
  const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int tile = 0; tile < 12; ++tile) {
    const int a = tile >> 2, sb = (tile & 3) * 8;
    const float *col = scr + (sb + g) * kTcRow + a * NC;  // segment sb + g, axis a
    const float x0 = col[t], x1 = col[t + 4];
    const uint32_t bh0 = tf32_rna(x0), bh1 = tf32_rna(x1);
    const uint32_t bl0 = tf32_rna(x0 - __uint_as_float(bh0)), bl1 = tf32_rna(x1 - __uint_as_float(bh1));
    float d[4];
    mma_tf32(d, A.hi0, A.lo0, A.hi1, A.lo1, bh0, bh1, zero);  // rows 0-7: G_hi B_hi, rows 8-15: G_lo B_hi
    mma_tf32(d, A.hi0, 0u, A.hi1, 0u, bl0, bl1, d);           // rows 0-7: + G_hi B_lo
    out[tile][0] = d[0] + d[2];
    out[tile][1] = d[1] + d[3];
  }
  __syncwarp();
#pragma unroll
  for (int tile = 0; tile < 12; ++tile) {
    const int a = tile >> 2, sb = (tile & 3) * 8;
    // D row g = coefficient g; columns 2t, 2t+1 = segments sb + 2t, sb + 2t + 1
    scr[(sb + 2 * t) * kTcRow + a * NC + g] = out[tile][0];
    scr[(sb + 2 * t + 1) * kTcRow + a * NC + g] = out[tile][1];
  }
  __syncwarp();
#pragma unroll
  for (int a = 0; a < AX; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) ch[a][k] = mine[a * NC + k];
  __syncwarp();
}

}  // namespace top
