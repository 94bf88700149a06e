// The learned component: a two-layer MLP with BF16 weights and activations
// and FP32 accumulation that proposes per-neuron ReLU orders (and, with
// another head size, split dimensions).  Kernels live in k_mlp.cu.
#pragma once

#include <cuda_bf16.h>

#include "bern_internal.cuh"

namespace bern {

constexpr int kMlpHidden = BERN_MLP_HIDDEN;
constexpr int kMlpMaxF = BERN_MLP_MAX_FEATURES;
constexpr int kMlpMaxC = BERN_MLP_MAX_CLASSES;
constexpr int kDegFeatures = BERN_DEGREE_FEATURES;
constexpr int kDegClasses = BERN_DEGREE_CLASSES;

struct MlpView {
  int F, C;
  const __nv_bfloat16* W1;   // [H x F]
  const float* b1;           // [H]
  const __nv_bfloat16* W2;   // [C x H]
  const float* b2;           // [C]
};

inline int64_t mlp_num_params(int F, int C) {
  return (int64_t)kMlpHidden * F + kMlpHidden + (int64_t)C * kMlpHidden + C;
}

// Scratch bytes of launch_mlp_backward for n samples.
size_t mlp_backward_scratch(int64_t n, int F, int C);

// The degree features of one item (the definition is in include/bern.h,
// bern_degree_features).
__device__ __forceinline__ void degree_feature_vec(float l, float h, int nt, int layer,
                                                   float (&o)[kDegFeatures]) {
  const float s = fmaxf(fmaxf(fabsf(l), fabsf(h)), 1e-30f);
  o[0] = l / s;
  o[1] = h / s;
  o[2] = log2f(fmaxf(h - l, 1e-30f)) * 0.125f;
  o[3] = (float)layer * 0.125f;
  o[4] = log2f((float)max(nt, 1)) * 0.0625f;
  o[5] = l >= 0.0f ? 1.0f : 0.0f;
  o[6] = h <= 0.0f ? 1.0f : 0.0f;
  o[7] = l >= 0.0f ? 0.0f : (h <= 0.0f ? 1.0f : fminf(1.0f, fmaxf(0.0f, -l / (h - l))));
}

// Learned plan, one hidden layer: per (box, neuron) the degree MLP's
// proposal d (class c -> order c + 1; the fallback order when the largest
// probability is below min_conf; at most max_d), the ReLU case and
// coefficients for d, and
// per box the next Bernstein order min(cap, order_in * max_m d).
cudaError_t launch_learned_degrees(const Launch& L, const MlpView& M, int64_t n_boxes, int h,
                                   int layer, const float* lo, const float* hi,
                                   const int32_t* pre_nterms, float min_conf, int fallback_d,
                                   int max_d, int cap, const int32_t* order_in,
                                   int32_t* order_out, uint8_t* degrees, int8_t* kind,
                                   float* coef, float* eps);
cudaError_t launch_fill_i32(const Launch& L, int32_t* p, int64_t n, int32_t v);

cudaError_t launch_degree_features(const Launch& L, int64_t n_items, const float* lo,
                                   const float* hi, const int32_t* nterms, int layer, float* x);
cudaError_t launch_mlp_forward(const Launch& L, const MlpView& M, int64_t n, const float* x,
                               float* logits);
cudaError_t launch_mlp_backward(const Launch& L, const MlpView& M, int64_t n, const float* x,
                                const int32_t* labels, const float* w, void* scratch,
                                float* grad, float* loss);
cudaError_t launch_mlp_adam(const Launch& L, int F, int C, float* param, float* m, float* v,
                            const float* grad, float lr, float beta1, float beta2, float eps,
                            float c1, float c2, __nv_bfloat16* W1b, __nv_bfloat16* W2b);

}  // namespace bern
