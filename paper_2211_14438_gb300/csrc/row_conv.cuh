// Row convolutions of the squaring step (a4, order 2): one output row of the
// square of a polynomial held in row layout (monomials sharing the exponents
// of t_1..t_{n-1} contiguous), as the sum of 1-D convolutions of input-row
// pairs, unrolled for every pair of row lengths up to kRowLen.  Shared by
// the composition kernel (k_compose.cu) and the fused layer kernel
// (k_layer.cu).
#pragma once

#include "device_util.cuh"

namespace bern {

// One accumulator per output slot holds the square directly: an off-diagonal
// row pair (p < q) counts twice in the square, so it multiplies 2*x[a]
// (exact) by y[b]; the diagonal pair (p == q) is the row's own square,
// sum_a x[a]^2 t^(2a) + sum_(a<b) 2 x[a] x[b] t^(a+b), taken as a triangle.
// Every product is accumulated with a directed FMA.
template <int L1, int L2, bool UP>
__device__ __forceinline__ void conv_rows(const float* __restrict__ s, int offp, int offq,
                                          float (&acc)[2 * kRowLen - 1]) {
  float x[L1], y[L2];
#pragma unroll
  for (int a = 0; a < L1; ++a) {
    const float v = s[offp + a];
    x[a] = v + v;
  }
#pragma unroll
  for (int b = 0; b < L2; ++b) y[b] = s[offq + b];
#pragma unroll
  for (int a = 0; a < L1; ++a)
#pragma unroll
    for (int b = 0; b < L2; ++b) acc[a + b] = dfma<UP>(x[a], y[b], acc[a + b]);
}

template <int L, bool UP>
__device__ __forceinline__ void conv_diag(const float* __restrict__ s, int off,
                                          float (&acc)[2 * kRowLen - 1]) {
  float x[L], x2[L];
#pragma unroll
  for (int a = 0; a < L; ++a) {
    x[a] = s[off + a];
    x2[a] = x[a] + x[a];
  }
#pragma unroll
  for (int a = 0; a < L; ++a) {
    acc[2 * a] = dfma<UP>(x[a], x[a], acc[2 * a]);
#pragma unroll
    for (int b = a + 1; b < L; ++b) acc[a + b] = dfma<UP>(x2[a], x[b], acc[a + b]);
  }
}

#define BERN_CC(L1, L2) \
  case row_pair_case(L1, L2): conv_rows<L1, L2, UP>(s, pr.x, pr.y, acc); break;
#define BERN_CONV_ALL_CASES                                                                     \
  BERN_CC(1, 1) BERN_CC(1, 2) BERN_CC(1, 3) BERN_CC(1, 4) BERN_CC(1, 5) BERN_CC(1, 6)          \
  BERN_CC(1, 7) BERN_CC(1, 8) BERN_CC(1, 9) BERN_CC(2, 2) BERN_CC(2, 3) BERN_CC(2, 4)          \
  BERN_CC(2, 5) BERN_CC(2, 6) BERN_CC(2, 7) BERN_CC(2, 8) BERN_CC(2, 9) BERN_CC(3, 3)          \
  BERN_CC(3, 4) BERN_CC(3, 5) BERN_CC(3, 6) BERN_CC(3, 7) BERN_CC(3, 8) BERN_CC(3, 9)          \
  BERN_CC(4, 4) BERN_CC(4, 5) BERN_CC(4, 6) BERN_CC(4, 7) BERN_CC(4, 8) BERN_CC(4, 9)          \
  BERN_CC(5, 5) BERN_CC(5, 6) BERN_CC(5, 7) BERN_CC(5, 8) BERN_CC(5, 9) BERN_CC(6, 6)          \
  BERN_CC(6, 7) BERN_CC(6, 8) BERN_CC(6, 9) BERN_CC(7, 7) BERN_CC(7, 8) BERN_CC(7, 9)          \
  BERN_CC(8, 8) BERN_CC(8, 9) BERN_CC(9, 9)
#define BERN_CD(L) \
  case L: conv_diag<L, UP>(s, pr.x, acc); break;
#define BERN_DIAG_CASES \
  BERN_CD(1) BERN_CD(2) BERN_CD(3) BERN_CD(4) BERN_CD(5) BERN_CD(6) BERN_CD(7) BERN_CD(8) BERN_CD(9)

// The same with a per-lane sign sg = +1 or -1 on the first operand and
// round-up FMAs only.  With sg = -1 every partial sum is the exact negation
// of the round-down one (RU(-x) = -RD(x) in IEEE arithmetic), so lanes that
// compute the lower bound (sg = -1) and lanes that compute the upper bound
// (sg = +1) run the same instructions and produce bit for bit the values of
// conv_rows<.., false> (negated) and conv_rows<.., true>.
template <int L1, int L2>
__device__ __forceinline__ void conv_rows_sg(const float* __restrict__ s, int offp, int offq,
                                             float sg2, float (&acc)[2 * kRowLen - 1]) {
  float x[L1], y[L2];
#pragma unroll
  for (int a = 0; a < L1; ++a) x[a] = s[offp + a] * sg2;   // +-2 s: exact
#pragma unroll
  for (int b = 0; b < L2; ++b) y[b] = s[offq + b];
#pragma unroll
  for (int a = 0; a < L1; ++a)
#pragma unroll
    for (int b = 0; b < L2; ++b) acc[a + b] = __fmaf_ru(x[a], y[b], acc[a + b]);
}

template <int L>
__device__ __forceinline__ void conv_diag_sg(const float* __restrict__ s, int off, float sg,
                                             float (&acc)[2 * kRowLen - 1]) {
  float x[L], xs[L], x2[L];
#pragma unroll
  for (int a = 0; a < L; ++a) {
    x[a] = s[off + a];
    xs[a] = x[a] * sg;
    x2[a] = xs[a] + xs[a];
  }
#pragma unroll
  for (int a = 0; a < L; ++a) {
    acc[2 * a] = __fmaf_ru(xs[a], x[a], acc[2 * a]);
#pragma unroll
    for (int b = a + 1; b < L; ++b) acc[a + b] = __fmaf_ru(x2[a], x[b], acc[a + b]);
  }
}

#define BERN_CCS(L1, L2) \
  case row_pair_case(L1, L2): conv_rows_sg<L1, L2>(s, pr.x, pr.y, sg2, acc); break;
#define BERN_CONV_SG_CASES                                                                     \
  BERN_CCS(1, 1) BERN_CCS(1, 2) BERN_CCS(1, 3) BERN_CCS(1, 4) BERN_CCS(1, 5) BERN_CCS(1, 6)    \
  BERN_CCS(1, 7) BERN_CCS(1, 8) BERN_CCS(1, 9) BERN_CCS(2, 2) BERN_CCS(2, 3) BERN_CCS(2, 4)    \
  BERN_CCS(2, 5) BERN_CCS(2, 6) BERN_CCS(2, 7) BERN_CCS(2, 8) BERN_CCS(2, 9) BERN_CCS(3, 3)    \
  BERN_CCS(3, 4) BERN_CCS(3, 5) BERN_CCS(3, 6) BERN_CCS(3, 7) BERN_CCS(3, 8) BERN_CCS(3, 9)    \
  BERN_CCS(4, 4) BERN_CCS(4, 5) BERN_CCS(4, 6) BERN_CCS(4, 7) BERN_CCS(4, 8) BERN_CCS(4, 9)    \
  BERN_CCS(5, 5) BERN_CCS(5, 6) BERN_CCS(5, 7) BERN_CCS(5, 8) BERN_CCS(5, 9) BERN_CCS(6, 6)    \
  BERN_CCS(6, 7) BERN_CCS(6, 8) BERN_CCS(6, 9) BERN_CCS(7, 7) BERN_CCS(7, 8) BERN_CCS(7, 9)    \
  BERN_CCS(8, 8) BERN_CCS(8, 9) BERN_CCS(9, 9)
#define BERN_CDS(L) \
  case L: conv_diag_sg<L>(s, pr.x, sg, acc); break;
#define BERN_DIAG_SG_CASES \
  BERN_CDS(1) BERN_CDS(2) BERN_CDS(3) BERN_CDS(4) BERN_CDS(5) BERN_CDS(6) BERN_CDS(7) BERN_CDS(8) \
  BERN_CDS(9)

}  // namespace bern
