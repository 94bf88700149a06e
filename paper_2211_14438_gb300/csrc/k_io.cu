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
  const int64_t g = std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_trace<<<(unsigned)g, 256, 0, L.stream>>>(n_boxes, h, n_hidden, off, lo, hi, nt, deg,
                                              global_d, tr);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
