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
// Work decomposition: one block per (box, tile of TM neurons); a thread owns
// one monomial r and keeps TM upper + TM lower accumulators in registers, so
// every input coefficient it loads feeds 2*TM FMAs.  Loads of consecutive r
// by consecutive threads are coalesced.
#include "device_util.cuh"

namespace bern {

template <int TM>
__global__ void __launch_bounds__(128)
k_affine(int h_out, int h_in, const float* __restrict__ W, const float* __restrict__ bias,
         const float* __restrict__ in_up, const float* __restrict__ in_lo, int64_t in_stride,
         const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
         float* __restrict__ out_lo, int64_t out_stride, int32_t* __restrict__ out_nterms,
         int* status) {
  extern __shared__ float smem[];
  float* sW = smem;                                  // TM x h_in
  int32_t* sN = reinterpret_cast<int32_t*>(sW + TM * h_in);
  __shared__ int sMax;
  const int64_t box = blockIdx.x;
  const int m0 = blockIdx.y * TM;
  if (threadIdx.x == 0) sMax = 0;
  __syncthreads();
  int mloc = 0;
  for (int j = threadIdx.x; j < h_in; j += blockDim.x) {
    int v = in_nterms[box * h_in + j];
    if (v < 0 || v > in_stride) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    sN[j] = v;
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if ((threadIdx.x & 31) == 0) atomicMax(&sMax, mloc);
  for (int idx = threadIdx.x; idx < TM * h_in; idx += blockDim.x) {
    int mm = idx / h_in, j = idx - mm * h_in;
    sW[idx] = (m0 + mm < h_out) ? W[(int64_t)(m0 + mm) * h_in + j] : 0.0f;
  }
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_stride) {
    if (threadIdx.x == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  const float* pu = in_up + box * h_in * in_stride;
  const float* pl = in_lo + box * h_in * in_stride;
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    float up[TM], lo[TM];
#pragma unroll
    for (int mm = 0; mm < TM; ++mm) {
      float b0 = (r == 0 && m0 + mm < h_out) ? bias[m0 + mm] : 0.0f;
      up[mm] = b0;
      lo[mm] = b0;
    }
    for (int j = 0; j < h_in; ++j) {
      float u = 0.0f, l = 0.0f;
      if (r < sN[j]) {
        u = pu[(int64_t)j * in_stride + r];
        l = pl[(int64_t)j * in_stride + r];
      }
#pragma unroll
      for (int mm = 0; mm < TM; ++mm) {
        const float w = sW[mm * h_in + j];
        const bool pos = w > 0.0f;
        up[mm] = __fmaf_ru(w, pos ? u : l, up[mm]);
        lo[mm] = __fmaf_rd(w, pos ? l : u, lo[mm]);
      }
    }
#pragma unroll
    for (int mm = 0; mm < TM; ++mm) {
      if (m0 + mm < h_out) {
        const int64_t o = (box * h_out + m0 + mm) * out_stride + r;
        out_up[o] = up[mm];
        out_lo[o] = lo[mm];
      }
    }
  }
  if (threadIdx.x < TM && m0 + (int)threadIdx.x < h_out)
    out_nterms[box * h_out + m0 + threadIdx.x] = M;
}

cudaError_t launch_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                          const float* W, const float* b, const float* in_up,
                          const float* in_lo, int64_t in_stride, const int32_t* in_nterms,
                          float* out_up, float* out_lo, int64_t out_stride,
                          int32_t* out_nterms) {
  constexpr int TM = 8;
  if (n_boxes == 0) return cudaSuccess;
  dim3 grid((unsigned)n_boxes, (unsigned)((h_out + TM - 1) / TM));
  size_t smem = (size_t)TM * h_in * sizeof(float) + (size_t)h_in * sizeof(int32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_affine<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_affine<TM><<<grid, 128, smem, L.stream>>>(h_out, h_in, W, b, in_up, in_lo, in_stride,
                                              in_nterms, out_up, out_lo, out_stride,
                                              out_nterms, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
