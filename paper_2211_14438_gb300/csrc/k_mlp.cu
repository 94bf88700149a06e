// The learned component's kernels: degree features, BF16 MLP inference,
// the cross-entropy gradient (deterministic two-pass reduction) and Adam.
//
// Forward, per sample (one thread), weights staged in shared memory:
//   xb = bf16(x);  for each hidden unit j:  z1_j = b1_j + sum_f W1_jf xb_f,
//   a_j = bf16(max(z1_j, 0)),  z_c += W2_cj a_j  (fp32 accumulation).
// Backward:  p = softmax(z),  dz_c = w (p_c - [c = y]),
//   dW2_cj = sum_s dz_c a_j,  db2_c = sum_s dz_c,
//   dz1_j = [z1_j > 0] sum_c W2_cj dz_c,  dW1_jf = sum_s dz1_j xb_f,  db1_j = sum_s dz1_j,
// all divided by n.  Per-sample terms go to scratch; a second kernel sums
// them per parameter over fixed chunks of samples and a third adds the chunk
// partials in chunk order, so the result does not depend on scheduling.
#include <math.h>

#include "device_util.cuh"
#include "enclose_impl.cuh"
#include "mlp.cuh"

namespace bern {

namespace {

constexpr int kH = kMlpHidden;
constexpr int kChunk = 1024;   // samples per partial sum

struct SmemMlp {
  float W1[kH * kMlpMaxF];     // [j][f], zero-padded to kMlpMaxF
  float b1[kH];
  float W2[kMlpMaxC * kH];     // [c][j]
  float b2[kMlpMaxC];
};

__device__ void stage_mlp(const MlpView& M, SmemMlp& S) {
  for (int i = threadIdx.x; i < kH * kMlpMaxF; i += blockDim.x) {
    const int j = i / kMlpMaxF, f = i % kMlpMaxF;
    S.W1[i] = f < M.F ? __bfloat162float(M.W1[j * M.F + f]) : 0.0f;
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) S.b1[i] = M.b1[i];
  for (int i = threadIdx.x; i < kMlpMaxC * kH; i += blockDim.x)
    S.W2[i] = i < M.C * kH ? __bfloat162float(M.W2[i]) : 0.0f;
  for (int i = threadIdx.x; i < kMlpMaxC; i += blockDim.x) S.b2[i] = i < M.C ? M.b2[i] : 0.0f;
  __syncthreads();
}

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__device__ __forceinline__ float hidden_pre(const SmemMlp& S, int j, const float (&xb)[kMlpMaxF]) {
  float acc = S.b1[j];
#pragma unroll
  for (int f = 0; f < kMlpMaxF; ++f) acc = fmaf(S.W1[j * kMlpMaxF + f], xb[f], acc);
  return acc;
}

// Logits of one sample; optionally stores the bf16 activations.
__device__ void mlp_logits(const SmemMlp& S, const float (&xb)[kMlpMaxF], float (&z)[kMlpMaxC],
                           __nv_bfloat16* a_out) {
#pragma unroll
  for (int c = 0; c < kMlpMaxC; ++c) z[c] = S.b2[c];
  for (int j = 0; j < kH; ++j) {
    const float a = bf16_round(fmaxf(hidden_pre(S, j, xb), 0.0f));
    if (a_out) a_out[j] = __float2bfloat16_rn(a);
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c) z[c] = fmaf(S.W2[c * kH + j], a, z[c]);
  }
}

__device__ void load_features(const float* x, int F, int64_t s, float (&xb)[kMlpMaxF]) {
#pragma unroll
  for (int f = 0; f < kMlpMaxF; ++f) xb[f] = f < F ? bf16_round(x[s * F + f]) : 0.0f;
}

__global__ void __launch_bounds__(128)
k_degree_features(int64_t n, const float* __restrict__ lo, const float* __restrict__ hi,
                  const int32_t* __restrict__ nterms, int layer, float* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f[kDegFeatures];
    degree_feature_vec(lo[i], hi[i], nterms ? nterms[i] : 1, layer, f);
#pragma unroll
    for (int k = 0; k < kDegFeatures; ++k) x[i * kDegFeatures + k] = f[k];
  }
}

// One block per box; threads over the box's neurons.
__global__ void __launch_bounds__(128)
k_learned_degrees(MlpView M, int64_t n_boxes, int h, int layer, const float* __restrict__ lo,
                  const float* __restrict__ hi, const int32_t* __restrict__ pre_nterms,
                  float min_conf, int fallback_d, int max_d, int cap,
                  const int32_t* __restrict__ order_in,
                  int32_t* __restrict__ order_out, uint8_t* __restrict__ degrees,
                  int8_t* __restrict__ kind, float* __restrict__ coef, float* __restrict__ eps,
                  int* status) {
  __shared__ SmemMlp S;
  __shared__ int s_max;
  stage_mlp(M, S);
  for (int64_t b = blockIdx.x; b < n_boxes; b += gridDim.x) {
    if (threadIdx.x == 0) s_max = 1;
    __syncthreads();
    int dmax = 1;
    for (int m = threadIdx.x; m < h; m += blockDim.x) {
      const int64_t it = b * h + m;
      const float l = lo[it], u = hi[it];
      float f[kDegFeatures], xb[kMlpMaxF], z[kMlpMaxC];
      degree_feature_vec(l, u, pre_nterms[it], layer, f);
#pragma unroll
      for (int k = 0; k < kMlpMaxF; ++k) xb[k] = k < kDegFeatures ? bf16_round(f[k]) : 0.0f;
      mlp_logits(S, xb, z, nullptr);
      int best = 0;
      float zb = z[0];
#pragma unroll
      for (int c = 1; c < kDegClasses; ++c)
        if (z[c] > zb) {   // first maximum wins ties
          zb = z[c];
          best = c;
        }
      float sum = 0.0f;
#pragma unroll
      for (int c = 0; c < kDegClasses; ++c) sum += expf(z[c] - zb);
      const float conf = 1.0f / sum;   // the largest softmax probability
      const int d = min(conf >= min_conf ? best + 1 : fallback_d, max_d);
      degrees[it] = (uint8_t)d;
      kind[it] = (int8_t)relu_item(l, u, d, coef + it * kCoefStride, eps + it, status);
      dmax = max(dmax, d);
    }
    dmax = warp_imax(dmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, dmax);
    __syncthreads();
    if (threadIdx.x == 0) order_out[b] = min(cap, order_in[b] * s_max);
    __syncthreads();
  }
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void __launch_bounds__(128)
k_mlp_forward(MlpView M, int64_t n, const float* __restrict__ x, float* __restrict__ logits) {
  __shared__ SmemMlp S;
  stage_mlp(M, S);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    float xb[kMlpMaxF], z[kMlpMaxC];
    load_features(x, M.F, s, xb);
    mlp_logits(S, xb, z, nullptr);
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c)
      if (c < M.C) logits[s * M.C + c] = z[c];
  }
}

struct BackScratch {
  float* dz1;            // [n][H]
  __nv_bfloat16* a;      // [n][H]
  float* dz2;            // [n][C]
  float* loss;           // [n]
  float* partial;        // [chunks][P + 1]
};

BackScratch carve(void* base, int64_t n, int C, int64_t P) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)base;
  BackScratch b;
  b.dz1 = (float*)p;
  p += al(sizeof(float) * n * kH);
  b.a = (__nv_bfloat16*)p;
  p += al(sizeof(__nv_bfloat16) * n * kH);
  b.dz2 = (float*)p;
  p += al(sizeof(float) * n * C);
  b.loss = (float*)p;
  p += al(sizeof(float) * n);
  b.partial = (float*)p;   // [chunks][P + 1]
  (void)P;
  return b;
}

__global__ void __launch_bounds__(128)
k_mlp_back_samples(MlpView M, int64_t n, const float* __restrict__ x,
                   const int32_t* __restrict__ labels, const float* __restrict__ w,
                   BackScratch B, int* status) {
  __shared__ SmemMlp S;
  stage_mlp(M, S);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    float xb[kMlpMaxF], z[kMlpMaxC];
    load_features(x, M.F, s, xb);
    mlp_logits(S, xb, z, B.a + s * kH);
    float mx = -INFINITY;
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c)
      if (c < M.C) mx = fmaxf(mx, z[c]);
    float e[kMlpMaxC], sum = 0.0f;
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c) {
      e[c] = c < M.C ? expf(z[c] - mx) : 0.0f;
      sum += e[c];
    }
    int y = labels[s];
    float ws = w ? w[s] : 1.0f;
    if (y < 0 || y >= M.C) {
      atomicOr(status, kStatusInvalid);
      y = 0;
      ws = 0.0f;
    }
    float zy = 0.0f;
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c)
      if (c == y) zy = z[c];
    B.loss[s] = ws * (logf(sum) - (zy - mx));
    float dz[kMlpMaxC];
    const float inv = 1.0f / sum;
#pragma unroll
    for (int c = 0; c < kMlpMaxC; ++c) {
      dz[c] = c < M.C ? ws * (e[c] * inv - (c == y ? 1.0f : 0.0f)) : 0.0f;
      if (c < M.C) B.dz2[s * M.C + c] = dz[c];
    }
    for (int j = 0; j < kH; ++j) {
      float dh = 0.0f;
#pragma unroll
      for (int c = 0; c < kMlpMaxC; ++c) dh = fmaf(S.W2[c * kH + j], dz[c], dh);
      B.dz1[s * kH + j] = hidden_pre(S, j, xb) > 0.0f ? dh : 0.0f;
    }
  }
}

// partial[chunk][p] for p < P (parameters) and p == P (loss)
__global__ void __launch_bounds__(128)
k_mlp_back_partials(int F, int C, int64_t n, const float* __restrict__ x, BackScratch B,
                    int64_t P) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  const int64_t s0 = (int64_t)blockIdx.y * kChunk, s1 = min(n, s0 + kChunk);
  const int64_t oW1 = (int64_t)kH * F, ob1 = oW1 + kH, oW2 = ob1 + (int64_t)C * kH;
  float acc = 0.0f;
  if (p < oW1) {
    const int j = (int)(p / F), f = (int)(p % F);
    for (int64_t s = s0; s < s1; ++s) acc = fmaf(B.dz1[s * kH + j], bf16_round(x[s * F + f]), acc);
  } else if (p < ob1) {
    const int j = (int)(p - oW1);
    for (int64_t s = s0; s < s1; ++s) acc += B.dz1[s * kH + j];
  } else if (p < oW2) {
    const int q = (int)(p - ob1), c = q / kH, j = q % kH;
    for (int64_t s = s0; s < s1; ++s)
      acc = fmaf(B.dz2[s * C + c], __bfloat162float(B.a[s * kH + j]), acc);
  } else if (p < P) {
    const int c = (int)(p - oW2);
    for (int64_t s = s0; s < s1; ++s) acc += B.dz2[s * C + c];
  } else {
    for (int64_t s = s0; s < s1; ++s) acc += B.loss[s];
  }
  B.partial[(int64_t)blockIdx.y * (P + 1) + p] = acc;
}

__global__ void __launch_bounds__(128)
k_mlp_back_final(int64_t n, int64_t P, int chunks, const float* __restrict__ partial,
                 float* __restrict__ grad, float* __restrict__ loss) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  float acc = 0.0f;
  for (int c = 0; c < chunks; ++c) acc += partial[(int64_t)c * (P + 1) + p];
  const float v = acc / (float)n;
  if (p < P)
    grad[p] = v;
  else
    loss[0] = v;
}

__global__ void __launch_bounds__(256)
k_mlp_adam(int F, int C, int64_t P, float* __restrict__ param, float* __restrict__ m,
           float* __restrict__ v, const float* __restrict__ grad, float lr, float beta1,
           float beta2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ W1b,
           __nv_bfloat16* __restrict__ W2b) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float g = grad[p];
  const float mm = beta1 * m[p] + (1.0f - beta1) * g;
  const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float th = param[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  param[p] = th;
  const int64_t oW1 = (int64_t)kH * F, ob1 = oW1 + kH, oW2 = ob1 + (int64_t)C * kH;
  if (p < oW1) W1b[p] = __float2bfloat16_rn(th);
  else if (p >= ob1 && p < oW2) W2b[p - ob1] = __float2bfloat16_rn(th);
}

int chunks_of(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }

}  // namespace

size_t mlp_backward_scratch(int64_t n, int F, int C) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t P = mlp_num_params(F, C);
  return al(sizeof(float) * n * kH) + al(2 * (size_t)n * kH) + al(sizeof(float) * n * C) +
         al(sizeof(float) * n) + al(sizeof(float) * (size_t)chunks_of(n) * (P + 1));
}

static unsigned grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)(g < cap ? g : cap);
}

cudaError_t launch_degree_features(const Launch& L, int64_t n_items, const float* lo,
                                   const float* hi, const int32_t* nterms, int layer, float* x) {
  if (n_items == 0) return cudaSuccess;
  k_degree_features<<<grid_for(n_items, 128, device_sms(L) * 32), 128, 0, L.stream>>>(n_items, lo, hi,
                                                                           nterms, layer, x);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_learned_degrees(const Launch& L, const MlpView& M, int64_t n_boxes, int h,
                                   int layer, const float* lo, const float* hi,
                                   const int32_t* pre_nterms, float min_conf, int fallback_d,
                                   int max_d, int cap, const int32_t* order_in,
                                   int32_t* order_out, uint8_t* degrees, int8_t* kind,
                                   float* coef, float* eps) {
  if (n_boxes == 0) return cudaSuccess;
  if (M.F != kDegFeatures || M.C != kDegClasses) return cudaErrorInvalidValue;
  k_learned_degrees<<<grid_for(n_boxes, 1, device_sms(L) * 16), 128, 0, L.stream>>>(
      M, n_boxes, h, layer, lo, hi, pre_nterms, min_conf, fallback_d, max_d, cap, order_in,
      order_out,
      degrees, kind, coef, eps, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_fill_i32(const Launch& L, int32_t* p, int64_t n, int32_t v) {
  if (n == 0) return cudaSuccess;
  k_fill_i32<<<grid_for(n, 256, device_sms(L) * 8), 256, 0, L.stream>>>(p, n, v);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const Launch& L, const MlpView& M, int64_t n, const float* x,
                               float* logits) {
  if (n == 0) return cudaSuccess;
  k_mlp_forward<<<grid_for(n, 128, device_sms(L) * 16), 128, 0, L.stream>>>(M, n, x, logits);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const Launch& L, const MlpView& M, int64_t n, const float* x,
                                const int32_t* labels, const float* w, void* scratch,
                                float* grad, float* loss) {
  if (n <= 0) return cudaErrorInvalidValue;
  const int64_t P = mlp_num_params(M.F, M.C);
  BackScratch B = carve(scratch, n, M.C, P);
  k_mlp_back_samples<<<grid_for(n, 128, device_sms(L) * 16), 128, 0, L.stream>>>(M, n, x, labels, w, B,
                                                                       L.status);
  const int chunks = chunks_of(n);
  dim3 g2((unsigned)((P + 1 + 127) / 128), (unsigned)chunks);
  k_mlp_back_partials<<<g2, 128, 0, L.stream>>>(M.F, M.C, n, x, B, P);
  k_mlp_back_final<<<(unsigned)((P + 1 + 127) / 128), 128, 0, L.stream>>>(n, P, chunks,
                                                                           B.partial, grad, loss);
  *L.launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const Launch& L, int F, int C, float* param, float* m, float* v,
                            const float* grad, float lr, float beta1, float beta2, float eps,
                            float c1, float c2, __nv_bfloat16* W1b, __nv_bfloat16* W2b) {
  const int64_t P = mlp_num_params(F, C);
  k_mlp_adam<<<(unsigned)((P + 255) / 256), 256, 0, L.stream>>>(F, C, P, param, m, v, grad, lr,
                                                                 beta1, beta2, eps, c1, c2, W1b,
                                                                 W2b);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
