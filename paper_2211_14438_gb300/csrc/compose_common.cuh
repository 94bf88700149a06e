// Shared definitions of the composition kernels (a4): the work-queue ids
// and the argument block of one composition call.
#pragma once

#include "device_util.cuh"

namespace bern {

constexpr float kU = 0x1p-24f;   // unit roundoff of float32
constexpr int kQIdent = kMaxRowDegree + 1;   // identity copies
constexpr int kQLinear = kMaxRowDegree + 2;  // order-1 items
constexpr int kQPairs = kMaxRowDegree + 3;   // order-2 items outside the row path
constexpr int kQHorner = kMaxRowDegree + 4;  // Horner items (order >= 3, or pruning)
static_assert(kQHorner + 1 == kComposeQueues, "queue ids");

struct ComposeArgs {
  int cap;
  float tau;                 // pruning threshold (relative to the L1 norm), 0 = off
  int h;                     // neurons per box; item = b*h + m
  const int8_t* kind;
  const float* coef;
  const float* eps;
  const uint8_t* degrees;
  int global_d;
  const float* lo;
  const float* hi;
  const float* pre_up;
  const float* pre_lo;
  int64_t pre_ld;
  const int32_t* pre_nterms;
  float* post_up;
  float* post_lo;
  int64_t post_ld;
  int32_t* post_nterms;
  // offset of coefficient 0 of an item in a block with leading dimension ld;
  // coefficient r is at offset + r*h
  __device__ __forceinline__ int64_t base(int64_t item, int64_t ld) const {
    const int64_t b = item / h;
    return (b * ld) * h + (item - b * h);
  }
};

__device__ __forceinline__ int degree_of(const Tables& T, int m) {
  if (m >= 0 && m <= T.mexps) return T.deg_of[m];
  int D = 0;
  while (D < kMaxTableDegree && T.mcount[D] < m) ++D;
  return D;
}

// The Horner kernel (k_horner.cu) over queue kQHorner, for inputs of degree
// <= Dmax and outputs of degree <= Dout (host functions; the sizes come from
// num_monomials, never from the device tables).
size_t horner_smem_floats(const Tables& T, int Dmax, int Dout);
// Global workspace floats (ComposeScratch::hws) the Horner kernel needs with
// `blocks` workspace slices, 0 when its buffers fit `smem_limit` bytes of
// shared memory.
size_t horner_global_floats(const Tables& T, int Dmax, int Dout, int64_t smem_limit, int blocks);
cudaError_t launch_compose_horner(const Launch& L, const Tables& T, const ComposeScratch& S,
                                  const ComposeArgs& A, int Dmax, int Dout);

}  // namespace bern
