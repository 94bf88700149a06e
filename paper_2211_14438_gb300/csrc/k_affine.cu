// a1: the layer step of Sec. 5.2 (eqs. upper_bounds_layer / lower_bounds_layer)
//
//   pre_up_m = b_m + sum_j W+_mj up_j + W-_mj lo_j
//   pre_lo_m = b_m + sum_j W+_mj lo_j + W-_mj up_j
//
// applied coefficient-wise over the shared graded monomial prefix.  The
// upper sum is accumulated with round-up FMAs and the lower one with
// round-down FMAs, so each computed coefficient bounds the exact one from the
// correct side; with t^K >= 0 on the box that bounds the polynomial values.
//
// With the layer-block layout (coefficient r of neuron j of box b at
// ((b*ld + r)*h + j)) each box is a row-major [M x h_in] matrix per bound and
// the step is the product with W^T: a small GEMM per box.  A block computes a
// BM (neurons) x BR (monomials) tile of one box; K (= h_in) is staged through
// shared memory in chunks of KC, and every thread keeps a TM x TR register
// tile per bound.  Inputs beyond a neuron's term count are read as zero.
#include <algorithm>

#include "device_util.cuh"

namespace bern {

template <int BM, int BR, int TM, int TR, int KC>
__global__ void __launch_bounds__((BM / TM) * (BR / TR))
k_affine(int h_out, int h_in, const float* __restrict__ W, const float* __restrict__ bias,
         const float* __restrict__ in_up, const float* __restrict__ in_lo, int64_t in_ld,
         const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
         float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
         int* status) {
  constexpr int NT = (BM / TM) * (BR / TR);
  constexpr int TX = BM / TM;                       // threads along m
  __shared__ float sW[KC][BM];
  __shared__ float sU[BR][KC + 1];
  __shared__ float sL[BR][KC + 1];
  __shared__ int sMax;
  extern __shared__ int32_t sN[];                   // h_in term counts
  const int64_t b = blockIdx.x;
  const int r0 = blockIdx.y * BR;
  const int m0 = blockIdx.z * BM;
  const int tid = threadIdx.x;
  if (tid == 0) sMax = 0;
  __syncthreads();
  int mloc = 0;
  for (int j = tid; j < h_in; j += NT) {
    int v = in_nterms[b * h_in + j];
    if (v < 0 || v > in_ld) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    sN[j] = v;
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if ((tid & 31) == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (tid == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0)
    for (int m = m0 + tid; m < min(m0 + BM, h_out); m += NT) out_nterms[b * h_out + m] = M;
  if (r0 >= M) return;

  const int tm = tid % TX, tr = tid / TX;
  float up[TM][TR], lo[TM][TR];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int k = 0; k < TR; ++k) {
      const int m = m0 + tm * TM + i, r = r0 + tr * TR + k;
      const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
      up[i][k] = b0;
      lo[i][k] = b0;
    }
  const float* gU = in_up + (b * in_ld) * h_in;
  const float* gL = in_lo + (b * in_ld) * h_in;
  for (int j0 = 0; j0 < h_in; j0 += KC) {
    // stage W[m0.., j0..] transposed, and the input rows r0.. of columns j0..
    for (int idx = tid; idx < KC * BM; idx += NT) {
      const int mm = idx % BM, jj = idx / BM;
      const int m = m0 + mm, j = j0 + jj;
      sW[jj][mm] = (m < h_out && j < h_in) ? W[(int64_t)m * h_in + j] : 0.0f;
    }
    for (int idx = tid; idx < KC * BR; idx += NT) {
      const int jj = idx % KC, rr = idx / KC;
      const int j = j0 + jj, r = r0 + rr;
      float u = 0.0f, l = 0.0f;
      if (j < h_in && r < sN[j]) {
        u = gU[(int64_t)r * h_in + j];
        l = gL[(int64_t)r * h_in + j];
      }
      sU[rr][jj] = u;
      sL[rr][jj] = l;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < KC; ++jj) {
      float w[TM], u[TR], l[TR];
#pragma unroll
      for (int i = 0; i < TM; ++i) w[i] = sW[jj][tm * TM + i];
#pragma unroll
      for (int k = 0; k < TR; ++k) {
        u[k] = sU[tr * TR + k][jj];
        l[k] = sL[tr * TR + k][jj];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const bool pos = w[i] > 0.0f;
#pragma unroll
        for (int k = 0; k < TR; ++k) {
          up[i][k] = __fmaf_ru(w[i], pos ? u[k] : l[k], up[i][k]);
          lo[i][k] = __fmaf_rd(w[i], pos ? l[k] : u[k], lo[i][k]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TR; ++k) {
    const int r = r0 + tr * TR + k;
    if (r >= M) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tm * TM + i;
      if (m < h_out) {
        const int64_t o = (b * out_ld + r) * h_out + m;
        out_up[o] = up[i][k];
        out_lo[o] = lo[i][k];
      }
    }
  }
}

// Narrow output layers (h_out <= 4, e.g. a network's output): one thread per
// (box, monomial row) reads its whole input row (contiguous over j) and
// keeps the HO outputs of both bounds in registers; no staging is needed.
template <int HO>
__global__ void __launch_bounds__(256)
k_affine_narrow(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
                const float* __restrict__ bias, const float* __restrict__ in_up,
                const float* __restrict__ in_lo, int64_t in_ld,
                const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
                float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
                int* status) {
  extern __shared__ float sW[];                      // h_out x h_in, then h_in counts
  int32_t* sN = reinterpret_cast<int32_t*>(sW + HO * h_in);
  __shared__ int sMax;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) sMax = 0;
  for (int i = threadIdx.x; i < HO * h_in; i += blockDim.x) {
    const int m = i / h_in;
    sW[i] = m < h_out ? W[i] : 0.0f;
  }
  __syncthreads();
  int mloc = 0;
  for (int j = threadIdx.x; j < h_in; j += blockDim.x) {
    int v = in_nterms[b * h_in + j];
    if (v < 0 || v > in_ld) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    sN[j] = v;
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if ((threadIdx.x & 31) == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (threadIdx.x == 0 && blockIdx.y == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0 && threadIdx.x < h_out) out_nterms[b * h_out + threadIdx.x] = M;
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= M) return;
  float up[HO], lo[HO];
#pragma unroll
  for (int m = 0; m < HO; ++m) {
    const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
    up[m] = b0;
    lo[m] = b0;
  }
  const float* pu = in_up + (b * in_ld + r) * h_in;
  const float* pl = in_lo + (b * in_ld + r) * h_in;
  auto step = [&](int j, float u, float l) {
    const bool live = r < sN[j];
    u = live ? u : 0.0f;
    l = live ? l : 0.0f;
#pragma unroll
    for (int m = 0; m < HO; ++m) {
      const float w = sW[m * h_in + j];
      const bool pos = w > 0.0f;
      up[m] = __fmaf_ru(w, pos ? u : l, up[m]);
      lo[m] = __fmaf_rd(w, pos ? l : u, lo[m]);
    }
  };
  if ((h_in & 3) == 0 && ((reinterpret_cast<uintptr_t>(pu) | reinterpret_cast<uintptr_t>(pl)) & 15) == 0) {
    // rows are 16-byte aligned: read them as float4
    const float4* pu4 = reinterpret_cast<const float4*>(pu);
    const float4* pl4 = reinterpret_cast<const float4*>(pl);
#pragma unroll 2
    for (int j4 = 0; j4 < (h_in >> 2); ++j4) {
      const float4 u = __ldg(pu4 + j4), l = __ldg(pl4 + j4);
      step(4 * j4, u.x, l.x);
      step(4 * j4 + 1, u.y, l.y);
      step(4 * j4 + 2, u.z, l.z);
      step(4 * j4 + 3, u.w, l.w);
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < h_in; ++j) step(j, __ldg(pu + j), __ldg(pl + j));
  }
#pragma unroll
  for (int m = 0; m < HO; ++m) {
    if (m < h_out) {
      const int64_t o = (b * out_ld + r) * h_out + m;
      out_up[o] = up[m];
      out_lo[o] = lo[m];
    }
  }
}

template <int BM, int BR, int TM, int TR, int KC>
static cudaError_t launch_cfg(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                              const float* W, const float* b, const float* in_up,
                              const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                              float* out_up, float* out_lo, int64_t out_ld,
                              int32_t* out_nterms) {
  // r tiles cover the largest possible term count (in_ld); tiles past a box's
  // actual count exit after the count is known
  const int64_t rt = (std::max<int64_t>(1, std::min(in_ld, out_ld)) + BR - 1) / BR;
  dim3 grid((unsigned)n_boxes, (unsigned)rt, (unsigned)((h_out + BM - 1) / BM));
  const size_t smem = (size_t)h_in * sizeof(int32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_affine<BM, BR, TM, TR, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_affine<BM, BR, TM, TR, KC><<<grid, (BM / TM) * (BR / TR), smem, L.stream>>>(
      h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld, out_nterms,
      L.status);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                          const float* W, const float* b, const float* in_up,
                          const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                          float* out_up, float* out_lo, int64_t out_ld,
                          int32_t* out_nterms) {
  if (n_boxes == 0) return cudaSuccess;
  if (n_boxes > 0x7fffffff || (std::min(in_ld, out_ld) + 15) / 16 > 65535)
    return cudaErrorInvalidValue;
  const bool few_rows = std::min(in_ld, out_ld) <= 16;     // short polynomials: short tiles
  if (h_out >= 32 && few_rows)
    return launch_cfg<64, 16, 4, 1, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  if (h_out >= 32)
    return launch_cfg<64, 64, 4, 4, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  if (h_out > 8 && few_rows)
    return launch_cfg<16, 16, 2, 1, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  if (h_out > 8)
    return launch_cfg<16, 64, 2, 4, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  // narrow outputs (h_out <= 8): a thread per monomial row, HO >= h_out
  const int HO = h_out == 1 ? 1 : (h_out <= 4 ? 4 : 8);
  const size_t smem = (size_t)HO * h_in * sizeof(float) + (size_t)h_in * sizeof(int32_t);
  const int64_t rows = std::max<int64_t>(1, std::min(in_ld, out_ld));
  if (smem > 200 * 1024 || (rows + 127) / 128 > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)n_boxes, (unsigned)((rows + 127) / 128));
  cudaError_t e = cudaSuccess;
#define BERN_NARROW(X)                                                                        \
  if (HO == X) {                                                                              \
    if (smem > 48 * 1024)                                                                     \
      e = cudaFuncSetAttribute(k_affine_narrow<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)smem);                                                    \
    if (e == cudaSuccess)                                                                     \
      k_affine_narrow<X><<<grid, 128, smem, L.stream>>>(n_boxes, h_out, h_in, W, b, in_up,    \
                                                        in_lo, in_ld, in_nterms, out_up,      \
                                                        out_lo, out_ld, out_nterms, L.status);\
  }
  BERN_NARROW(1)
  BERN_NARROW(4)
  BERN_NARROW(8)
#undef BERN_NARROW
  if (e != cudaSuccess) return e;
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
