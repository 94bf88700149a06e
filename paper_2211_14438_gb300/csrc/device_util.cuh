// Device helpers: directed rounding, block reductions, binomial tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bern_internal.cuh"

namespace bern {

// UP = round towards +inf (upper bounds), !UP = towards -inf (lower bounds)
template <bool UP>
__device__ __forceinline__ float dfma(float a, float b, float c) {
  return UP ? __fmaf_ru(a, b, c) : __fmaf_rd(a, b, c);
}
template <bool UP>
__device__ __forceinline__ float dadd(float a, float b) {
  return UP ? __fadd_ru(a, b) : __fadd_rd(a, b);
}

// warp-wide directed sum (fixed tree: deterministic)
template <bool UP>
__device__ __forceinline__ float warp_dsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dadd<UP>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_imax(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide directed sum; scratch holds >= 32 floats; all threads get the
// result.  Must be called by every thread of the block.
template <bool UP>
__device__ float block_dsum(float v, float* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_dsum<UP>(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  float r = lane < nw ? scratch[lane] : 0.0f;
  r = warp_dsum<UP>(r);
  return r;
}

// Exact binomials C(l,k), l,k <= 24 (all < 2^24, so exact in float32).
struct BinomTable {
  float v[kMaxEncloseOrder + 1][kMaxEncloseOrder + 1];
};
constexpr BinomTable make_binom_table() {
  BinomTable t{};
  for (int l = 0; l <= kMaxEncloseOrder; ++l) {
    t.v[l][0] = 1.0f;
    for (int k = 1; k <= l; ++k) t.v[l][k] = t.v[l - 1][k - 1] + (k <= l - 1 ? t.v[l - 1][k] : 0.0f);
  }
  return t;
}
__constant__ const BinomTable c_binom = make_binom_table();

__device__ __forceinline__ float binomf(int l, int k) { return c_binom.v[l][k]; }


}  // namespace bern
