// Shared definitions of the composition kernels (a4): the work-queue ids
// and the argument block of one composition call.
#pragma once

#include "device_util.cuh"

namespace bern {

constexpr float kU = 0x1p-24f;   // unit roundoff of float32
constexpr int kQIdent = kMaxRowDegree + 1;   // identity copies
constexpr int kQLinear = kMaxRowDegree + 2;  // order-1 items
constexpr int kQPairs = kMaxRowDegree + 3;   // order-2 items outside the row path
constexpr int kQHorner = kMaxRowDegree + 4;  // Horner items in float32 (order >= 3, or pruning)
constexpr int kQHorner64 = kMaxRowDegree + 5;  // Horner items in float64 (order >= kHornerF64Order)
static_assert(kQHorner64 + 1 == kComposeQueues, "queue ids");
// From this ReLU order on the composition runs in float64: the power-form
// coefficients of the order-d ReLU polynomial grow like C(d, d/2) 2^(d/2)
// (hi - lo) / d while the composed result stays of the order of hi - lo, so
// float32 rounding of the intermediate coefficients (u times their size)
// swamps the result's own accuracy at about this order.
constexpr int kHornerF64Order = 6;

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
  int64_t pre_cap;           // largest input term count (<= pre_ld)
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

// The Horner kernels (k_horner.cu) over queues kQHorner (float32) and
// kQHorner64 (float64), for inputs of degree <= Dmax, ReLU orders <= d and
// total-degree cap `cap` (host functions; the sizes come from
// num_monomials, never from the device tables).  Buffer floats per block
// (the larger of the two variants; float64 elements count as two floats).
size_t horner_smem_floats(const Tables& T, int Dmax, int cap, int d);
// Global workspace floats (ComposeScratch::hws) the Horner kernels need with
// `blocks` workspace slices, 0 when their buffers fit `smem_limit` bytes of
// shared memory (at most 200 KB).
size_t horner_global_floats(const Tables& T, int Dmax, int cap, int d, int64_t smem_limit,
                            int blocks);
// Launches the float32 kernel when its queue can be non-empty and the
// float64 one when A.global_d >= kHornerF64Order.
cudaError_t launch_compose_horner(const Launch& L, const Tables& T, const ComposeScratch& S,
                                  const ComposeArgs& A, int Dmax);

}  // namespace bern
