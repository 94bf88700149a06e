// a0 (input init, Sec. 5.3) and a5 (output copy-out).
//
// a0: the paper initialises x_i as the order-1 Bernstein tensor
// [dlo_i, dhi_i] (x) [1,1] (x) ... ; in the power basis of
// t_i = (x_i - dlo_i)/w_i that is the polynomial dlo_i + w_i t_i.  The width
// is rounded up (w_i >= dhi_i - dlo_i), so t in [0,1]^n covers the whole box.
// Layer-block layout: coefficient r of neuron i of box b at ((b*ld + r)*n + i).
#include <algorithm>

#include "device_util.cuh"

namespace bern {

__global__ void k_init_inputs(int n, int64_t n_boxes, const float* __restrict__ boxes,
                              float* __restrict__ z_up, float* __restrict__ z_lo, int64_t ld,
                              int32_t* __restrict__ nterms, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_boxes * n) return;
  const int64_t b = i / n;
  const int v = (int)(i - b * n);
  const float dl = boxes[2 * i], dh = boxes[2 * i + 1];
  float w = __fsub_ru(dh, dl);
  if (!(isfinite(dl) && isfinite(dh) && dl <= dh)) {
    atomicOr(status, kStatusInvalid);
    w = 0.0f;
  }
  for (int r = 0; r <= n; ++r) {
    const float c = r == 0 ? dl : (r == v + 1 ? w : 0.0f);
    const int64_t o = (b * ld + r) * n + v;
    z_up[o] = c;
    z_lo[o] = c;
  }
  nterms[i] = n + 1;
}

cudaError_t launch_init_inputs(const Launch& L, int n, int64_t n_boxes, const float* boxes,
                               float* z_up, float* z_lo, int64_t ld, int32_t* nterms) {
  if (n_boxes == 0) return cudaSuccess;
  const int64_t total = n_boxes * n;
  k_init_inputs<<<(unsigned)((total + 127) / 128), 128, 0, L.stream>>>(
      n, n_boxes, boxes, z_up, z_lo, ld, nterms, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// a5: copy the output-layer polynomials into the caller's (keys, coef) form.
// One block per (box, output).
__global__ void k_pack(Tables T, int o, const float* __restrict__ pre_up,
                       const float* __restrict__ pre_lo, int64_t ld,
                       const int32_t* __restrict__ nterms, bern_result res, int* status) {
  const int64_t item = blockIdx.x;
  const int64_t b = item / o;
  const int j = (int)(item - b * o);
  const int nt = nterms[item];
  if (threadIdx.x == 0) {
    res.n_terms[item * 2] = nt;
    res.n_terms[item * 2 + 1] = nt;
    if (nt > res.cap_terms && (res.coef || res.keys)) atomicOr(status, kStatusCapacity);
  }
  if (nt > res.cap_terms) return;
  const int n = T.n;
  for (int k = 0; k < 2; ++k) {
    const float* P = k == 0 ? pre_up : pre_lo;
    const int64_t base = (item * 2 + k) * res.cap_terms;
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
      if (res.coef) res.coef[base + r] = P[(b * ld + r) * o + j];
      if (res.keys) {
        uint64_t key = 0;
        for (int v = 0; v < n; ++v) key |= (uint64_t)T.exps[(int64_t)r * n + v] << (8 * v);
        res.keys[base + r] = key;
      }
    }
  }
}

cudaError_t launch_pack(const Launch& L, const Tables& T, int64_t n_boxes, int o,
                        const float* pre_up, const float* pre_lo, int64_t ld,
                        const int32_t* nterms, bern_result res) {
  if (n_boxes == 0) return cudaSuccess;
  k_pack<<<(unsigned)(n_boxes * o), 128, 0, L.stream>>>(T, o, pre_up, pre_lo, ld, nterms, res,
                                                        L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------ trace
__global__ void k_trace(int64_t n_boxes, int h, int64_t n_hidden, int64_t off,
                        const float* __restrict__ lo, const float* __restrict__ hi,
                        const int32_t* __restrict__ nt, const uint8_t* __restrict__ deg,
                        int global_d, bern_trace tr) {
  const int64_t n = n_boxes * h;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / h, m = i - b * h;
    const int64_t o = b * n_hidden + off + m;
    if (tr.lo) tr.lo[o] = lo[i];
    if (tr.hi) tr.hi[o] = hi[i];
    if (tr.nterms) tr.nterms[o] = nt[i];
    if (tr.degree) tr.degree[o] = deg ? deg[i] : (uint8_t)global_d;
  }
}

cudaError_t launch_trace(const Launch& L, int64_t n_boxes, int h, int64_t n_hidden, int64_t off,
                         const float* lo, const float* hi, const int32_t* nt,
                         const uint8_t* deg, int global_d, const bern_trace& tr) {
  const int64_t n = n_boxes * h;
  if (n == 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((n + 255) / 256, device_sms(L) * 8);
  k_trace<<<(unsigned)g, 256, 0, L.stream>>>(n_boxes, h, n_hidden, off, lo, hi, nt, deg,
                                              global_d, tr);
  ++*L.launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------ split features
// One block per box.  Features of output `j` (see bern_split_features).
__global__ void __launch_bounds__(128)
k_split_features(Tables T, int64_t n_boxes, int o, int j, const float* __restrict__ boxes,
                 const float* __restrict__ root, bern_result res, float* __restrict__ x,
                 int* status) {
  __shared__ float s_part[4][kMaxVars + 1];
  const int n = T.n, F = 2 * n + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < n_boxes; b += gridDim.x) {
    const int64_t p = (b * o + j) * 2;
    int ntu = res.n_terms[p], ntl = res.n_terms[p + 1];
    if (ntu < 0 || ntl < 0 || ntu > res.cap_terms || ntl > res.cap_terms || ntu > T.mexps ||
        ntl > T.mexps) {
      if (threadIdx.x == 0) atomicOr(status, kStatusInvalid);
      ntu = ntl = 0;
    }
    const float* cu = res.coef + p * res.cap_terms;
    const float* cl = cu + res.cap_terms;
    float sk[kMaxVars + 1];
#pragma unroll
    for (int k = 0; k <= kMaxVars; ++k) sk[k] = 0.0f;
    for (int r = threadIdx.x; r < max(ntu, ntl); r += blockDim.x) {
      const float u = r < ntu ? cu[r] : 0.0f, l = r < ntl ? cl[r] : 0.0f;
      sk[kMaxVars] += fabsf(u - l);
      const uint8_t* e = T.exps + (int64_t)r * n;
#pragma unroll
      for (int k = 0; k < kMaxVars; ++k)
        if (k < n) sk[k] += fabsf(u) * (float)e[k];
    }
#pragma unroll
    for (int k = 0; k <= kMaxVars; ++k) {
      float v = sk[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) s_part[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot[kMaxVars + 1];
      for (int k = 0; k <= kMaxVars; ++k)
        tot[k] = s_part[0][k] + s_part[1][k] + s_part[2][k] + s_part[3][k];
      float ssum = 0.0f;
      for (int k = 0; k < n; ++k) ssum += tot[k];
      float* xo = x + b * F;
      for (int k = 0; k < n; ++k) {
        const float side = boxes[(b * n + k) * 2 + 1] - boxes[(b * n + k) * 2];
        const float rside = root[k * 2 + 1] - root[k * 2];
        xo[k] = log2f(fmaxf(side, 1e-30f) / fmaxf(rside, 1e-30f)) * 0.0625f;
        xo[n + k] = tot[k] / fmaxf(ssum, 1e-30f);
      }
      xo[2 * n] = log2f(fmaxf(res.hi[b * o + j] - res.lo[b * o + j], 1e-30f)) * 0.125f;
      xo[2 * n + 1] = log2f(fmaxf(tot[kMaxVars], 1e-30f)) * 0.125f;
    }
    __syncthreads();
  }
}

cudaError_t launch_split_features(const Launch& L, const Tables& T, int64_t n_boxes, int o, int j,
                                  const float* boxes, const float* root, const bern_result& res,
                                  float* x) {
  if (n_boxes == 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>(n_boxes, device_sms(L) * 16);
  k_split_features<<<g, 128, 0, L.stream>>>(T, n_boxes, o, j, boxes, root, res, x, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
