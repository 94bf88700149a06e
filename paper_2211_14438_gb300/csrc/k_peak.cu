// FP32 FMA throughput of the device, measured: the denominator of the
// arithmetic rooflines of the kernels whose time goes to fused multiply-adds
// on the CUDA cores (affine, enclosure, composition).  Every thread runs
// kChains independent FMA chains, so the issue of the FMA pipe, not the
// latency of one chain, limits the rate; the grid fills every multiprocessor
// with kPeakBlocksPerSM blocks.  Directed rounding (round-up FMAs, as the
// bound kernels use) and round-to-nearest are measured separately.
#include <cuda_runtime.h>

#include <algorithm>

#include "bern_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 4;

// a value the compiler cannot predict keeps the chains alive
__device__ float g_peak_sink;

template <bool DIRECTED>
__global__ void __launch_bounds__(kPeakThreads)
k_fma_rate(int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = DIRECTED ? __fmaf_ru(a[i], m, c) : __fmaf_rn(a[i], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.0f) g_peak_sink = s;     // never true for these inputs
}

}  // namespace

extern "C" int bern_fma_throughput(int device, void* stream_handle, int directed, int reps,
                                  double* tflops) {
  if (!tflops || reps < 1) return BERN_E_INVALID;
  *tflops = 0.0;
  if (cudaSetDevice(device) != cudaSuccess) return BERN_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return BERN_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream_handle;
  const int blocks = sms * kPeakBlocksPerSM;
  const int iters = 1 << 16;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BERN_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BERN_E_CUDA;
  }
  float best = -1.0f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r = 0 warms up
    cudaEventRecord(e0, st);
    if (directed)
      k_fma_rate<true><<<blocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f);
    else
      k_fma_rate<false><<<blocks, kPeakThreads, 0, st>>>(iters, 0.999f, 1e-3f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.0f && (best < 0.0f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || best <= 0.0f) return BERN_E_CUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kPeakThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return BERN_OK;
}
