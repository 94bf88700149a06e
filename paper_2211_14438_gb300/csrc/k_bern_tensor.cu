// The paper's own representation on the GPU, for comparison with the power
// basis: the square of a polynomial held as a dense Bernstein tensor of
// order l in every variable (Sec. 4.1), by Prod_Bern (Sec. 4.2):
//
//   c_K = [ sum_{I+J=K} (a_I C_l(I)) (a_J C_l(J)) ] / C_2l(K),
//   C_l(I) = prod_k C(l, i_k),
//
// the Bernstein tensor of the square at order 2l (scale by the binomial
// tensors, multiply as power series, i.e. the full n-dimensional convolution,
// unscale).  One block per polynomial: the scaled tensor in shared memory,
// the threads over the output cells K, each summing over the box of I with
// max(0, k_j - l) <= i_j <= min(k_j, l).  The sums run in round-to-nearest
// beside the sum of the terms' magnitudes; an a-posteriori bound of every
// rounding on the way (the scaling products, the term products, the m-term
// sum, the binomial and the division) widens each coefficient to an
// interval [c_lo, c_hi] that contains the exact one.
#include <cuda_runtime.h>

#include <algorithm>

#include "compose_common.cuh"

namespace bern {

namespace {

constexpr int kBtThreads = 256;
constexpr int kBtMaxVars = 4;
constexpr int kBtMaxOrder = 8;

__device__ __forceinline__ float binom_l(int l, int k) { return binomf(l, k); }

__global__ void __launch_bounds__(kBtThreads)
k_bern_square(int n, int l, int64_t n_polys, const float* __restrict__ a, float* __restrict__ c_hi,
              float* __restrict__ c_lo, int* status) {
  extern __shared__ float su[];                 // (l+1)^n scaled coefficients
  const int R = l + 1, Ro = 2 * l + 1;
  int G = 1, Go = 1;
  for (int k = 0; k < n; ++k) {
    G *= R;
    Go *= Ro;
  }
  for (int64_t p = blockIdx.x; p < n_polys; p += gridDim.x) {
    const float* ap = a + p * G;
    for (int g = threadIdx.x; g < G; g += kBtThreads) {
      int rest = g;
      float w = 1.0f;
      for (int k = n - 1; k >= 0; --k) {
        w *= binom_l(l, rest % R);              // C(l, i) <= C(8,4) = 70: the product of
        rest /= R;                              // up to four is < 2^24, exact in float
      }
      su[g] = __fmul_rn(ap[g], w);
    }
    __syncthreads();
    for (int K = threadIdx.x; K < Go; K += kBtThreads) {
      int kd[kBtMaxVars], lo[kBtMaxVars], hi[kBtMaxVars], id[kBtMaxVars];
      int rest = K;
      float ck = 1.0f;
      for (int k = n - 1; k >= 0; --k) {
        kd[k] = rest % Ro;
        rest /= Ro;
        lo[k] = max(0, kd[k] - l);
        hi[k] = min(kd[k], l);
        id[k] = lo[k];
        ck *= binom_l(2 * l, kd[k]);            // rounded: C(16,8)^n exceeds 2^24
      }
      float s = 0.0f, m = 0.0f;
      int terms = 0;
      for (;;) {
        int gi = 0, gj = 0;
        for (int k = 0; k < n; ++k) {
          gi = gi * R + id[k];
          gj = gj * R + (kd[k] - id[k]);
        }
        const float x = su[gi], y = su[gj];
        s = __fmaf_rn(x, y, s);
        m = __fmaf_rn(fabsf(x), fabsf(y), m);
        ++terms;
        int k = n - 1;                          // odometer over the box of I
        while (k >= 0 && id[k] == hi[k]) {
          id[k] = lo[k];
          --k;
        }
        if (k < 0) break;
        ++id[k];
      }
      // |s - exact numerator| <= gamma_(terms+4) * sum |terms| (the two scaled
      // factors, the product and the terms-1 additions), and the computed m
      // underestimates that sum by at most the same factor; the binomial
      // product ck carries n roundings.  gamma_k = k u / (1 - k u), with k
      // taken as terms + 2n + 6 to cover all of them.
      const float ku = (float)(terms + 2 * n + 6) * kU;
      const float gamma = __fdiv_ru(ku, __fsub_rd(1.0f, ku));
      const float err = __fmul_ru(gamma, __fmul_ru(m, __fadd_ru(1.0f, gamma)));
      const float c_min = __fmul_rd(ck, __fsub_rd(1.0f, gamma));   // <= the exact C_2l(K)
      const float c_max = __fmul_ru(ck, __fadd_ru(1.0f, gamma));   // >= it
      const float nh = __fadd_ru(s, err), nl = __fsub_rd(s, err);
      // dividing by the smaller divisor moves a positive numerator up and a
      // negative one down
      const float hi2 = nh >= 0.0f ? __fdiv_ru(nh, c_min) : __fdiv_ru(nh, c_max);
      const float lo2 = nl <= 0.0f ? __fdiv_rd(nl, c_min) : __fdiv_rd(nl, c_max);
      c_hi[p * Go + K] = hi2;
      c_lo[p * Go + K] = lo2;
      if (!isfinite(hi2) || !isfinite(lo2)) atomicOr(status, kStatusNonFinite);
    }
    __syncthreads();
  }
}

}  // namespace

// The binomial weights of the scaling stay exact in float: (max_k C(l,k))^n < 2^24.
bool bernstein_square_ok(int n, int l) {
  if (n < 1 || n > kBtMaxVars || l < 0 || l > kBtMaxOrder) return false;
  double w = 1.0;
  for (int k = 0; k < n; ++k) {
    double c = 1.0;
    for (int i = 1; i <= l / 2; ++i) c = c * (l - l / 2 + i) / i;
    w *= c;
  }
  return w < 16777216.0;
}

cudaError_t launch_bernstein_square(const Launch& L, int n, int l, int64_t n_polys,
                                    const float* a, float* c_hi, float* c_lo) {
  if (n_polys == 0) return cudaSuccess;
  if (!bernstein_square_ok(n, l) || n_polys < 0) return cudaErrorInvalidValue;
  int G = 1;
  for (int k = 0; k < n; ++k) G *= l + 1;
  const size_t smem = (size_t)G * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bern_square, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = std::min<int64_t>(n_polys, (int64_t)device_sms(L) * 8);
  k_bern_square<<<(unsigned)blocks, kBtThreads, smem, L.stream>>>(n, l, n_polys, a, c_hi, c_lo,
                                                                   L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
