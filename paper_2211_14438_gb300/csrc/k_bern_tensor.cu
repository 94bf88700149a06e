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
// a thread per output row along the last variable, which adds the 1-D
// convolutions of every pair of input rows whose prefixes sum to its own
// (register-blocked, compile-time row length).  The sums run in round-to-nearest
// beside the sum of the terms' magnitudes; an a-posteriori bound of every
// rounding on the way (the scaling products, the term products, the m-term
// sum, the binomial and the division) widens each coefficient to an
// interval [c_lo, c_hi] that contains the exact one.
//
// Sum_Bern (Sec. 4.3) needs both operands at one order: degree elevation of
// a tensor from order l to l + r in every variable,
//
//   c'_k = sum_j c_j C(l, j) C(r, k - j) / C(l + r, k)     (per variable),
//
// one pass per variable with positive weights (exact float integers for
// l + r <= 24; the division by a bracket of the reciprocal), so round-up
// passes of an upper tensor and round-down passes of a lower one bound the
// exact elevation from the correct side; and the
// sum over a layer's neurons, b_m + sum_j W_mj c_j, which in the Bernstein
// basis adds the bias to every coefficient (the basis sums to one): the
// affine step's kernels on the tensors' coefficients, then the bias on the
// coefficients past the first.
#include <cuda_runtime.h>

#include <algorithm>

#include "compose_common.cuh"

namespace bern {

namespace {

constexpr int kBtMaxThreads = 512;
constexpr int kBtMaxVars = 4;
constexpr int kBtMaxOrder = 8;

__device__ __forceinline__ float binom_l(int l, int k) { return binomf(l, k); }

// One thread per output row (the 2L+1 cells that differ only in the last
// variable): for every pair of input rows whose prefixes add up to the output
// row's prefix, the 1-D convolution of the two rows (compile-time length
// L+1) into the row's accumulators, beside the same convolution of the
// magnitudes.  The tensor of the polynomial is scaled once per block.
template <int L>
__global__ void __launch_bounds__(kBtMaxThreads)
k_bern_square(int n, int64_t n_polys, const float* __restrict__ a, float* __restrict__ c_hi,
              float* __restrict__ c_lo, int* status) {
  extern __shared__ float su[];                 // (L+1)^n scaled coefficients
  constexpr int R = L + 1, Ro = 2 * L + 1;
  int G = 1, Go = 1, rows_out = 1;
  for (int k = 0; k < n; ++k) {
    G *= R;
    Go *= Ro;
  }
  rows_out = Go / Ro;
  // the largest number of products one output cell sums (a bound for the
  // a-posteriori error): (L+1)^n
  const float ku = (float)(G + 2 * n + 6) * kU;
  const float gamma = __fdiv_ru(ku, __fsub_rd(1.0f, ku));
  for (int64_t p = blockIdx.x; p < n_polys; p += gridDim.x) {
    const float* ap = a + p * G;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      int rest = g;
      float w = 1.0f;
      for (int k = n - 1; k >= 0; --k) {
        w *= binom_l(L, rest % R);              // exact: (max_k C(L,k))^n < 2^24
        rest /= R;
      }
      su[g] = __fmul_rn(ap[g], w);
    }
    __syncthreads();
    for (int orow = threadIdx.x; orow < rows_out; orow += blockDim.x) {
      int kd[kBtMaxVars], lo[kBtMaxVars], hi[kBtMaxVars], id[kBtMaxVars];
      int rest = orow;
      float ck_row = 1.0f;
      const int np = n - 1;                     // prefix digits (variables 1..n-1)
      for (int k = np - 1; k >= 0; --k) {
        kd[k] = rest % Ro;
        rest /= Ro;
        lo[k] = max(0, kd[k] - L);
        hi[k] = min(kd[k], L);
        id[k] = lo[k];
        ck_row *= binom_l(2 * L, kd[k]);        // rounded: C(2L, .)^n can exceed 2^24
      }
      float acc[Ro], mag[Ro];
#pragma unroll
      for (int c = 0; c < Ro; ++c) {
        acc[c] = 0.0f;
        mag[c] = 0.0f;
      }
      for (;;) {
        int ri = 0, rj = 0;
        for (int k = 0; k < np; ++k) {
          ri = ri * R + id[k];
          rj = rj * R + (kd[k] - id[k]);
        }
        float x[R], y[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          x[t] = su[ri * R + t];
          y[t] = su[rj * R + t];
        }
#pragma unroll
        for (int u = 0; u < R; ++u)
#pragma unroll
          for (int v = 0; v < R; ++v) {
            acc[u + v] = __fmaf_rn(x[u], y[v], acc[u + v]);
            mag[u + v] = __fmaf_rn(fabsf(x[u]), fabsf(y[v]), mag[u + v]);
          }
        int k = np - 1;                         // odometer over the prefix box
        while (k >= 0 && id[k] == hi[k]) {
          id[k] = lo[k];
          --k;
        }
        if (k < 0) break;
        ++id[k];
      }
      // |acc - exact numerator| <= gamma_(terms+4) sum |terms| and the computed
      // mag falls short of that sum by at most the same factor; the binomials
      // carry n roundings; gamma uses (L+1)^n + 2n + 6 >= all of them
#pragma unroll
      for (int c = 0; c < Ro; ++c) {
        const float ck = ck_row * binom_l(2 * L, c);
        const float err = __fmul_ru(gamma, __fmul_ru(mag[c], __fadd_ru(1.0f, gamma)));
        const float c_min = __fmul_rd(ck, __fsub_rd(1.0f, gamma));   // <= the exact C_2L(K)
        const float c_max = __fmul_ru(ck, __fadd_ru(1.0f, gamma));   // >= it
        const float nh = __fadd_ru(acc[c], err), nl = __fsub_rd(acc[c], err);
        // a smaller divisor moves a positive numerator up, a negative one down
        const float hv = nh >= 0.0f ? __fdiv_ru(nh, c_min) : __fdiv_ru(nh, c_max);
        const float lv = nl <= 0.0f ? __fdiv_rd(nl, c_min) : __fdiv_rd(nl, c_max);
        const int64_t K = p * Go + (int64_t)orow * Ro + c;
        c_hi[K] = hv;
        c_lo[K] = lv;
        if (!isfinite(hv) || !isfinite(lv)) atomicOr(status, kStatusNonFinite);
      }
    }
    __syncthreads();
  }
}

template <int L>
cudaError_t launch_l(const Launch& L_, int n, int64_t n_polys, const float* a, float* c_hi,
                     float* c_lo) {
  int G = 1;
  for (int k = 0; k < n; ++k) G *= L + 1;
  const size_t smem = (size_t)G * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bern_square<L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // a thread per output row: (2L+1)^(n-1) rows, rounded up to whole warps
  int rows = 1;
  for (int k = 0; k < n - 1; ++k) rows *= 2 * L + 1;
  const int threads = std::min(kBtMaxThreads, std::max(32, (rows + 31) & ~31));
  const int64_t blocks = std::min<int64_t>(n_polys, (int64_t)device_sms(L_) * 16);
  k_bern_square<L><<<(unsigned)blocks, threads, smem, L_.stream>>>(n, n_polys, a, c_hi, c_lo,
                                                                   L_.status);
  ++*L_.launches;
  return cudaGetLastError();
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
  switch (l) {
    case 0: return launch_l<0>(L, n, n_polys, a, c_hi, c_lo);
    case 1: return launch_l<1>(L, n, n_polys, a, c_hi, c_lo);
    case 2: return launch_l<2>(L, n, n_polys, a, c_hi, c_lo);
    case 3: return launch_l<3>(L, n, n_polys, a, c_hi, c_lo);
    case 4: return launch_l<4>(L, n, n_polys, a, c_hi, c_lo);
    case 5: return launch_l<5>(L, n, n_polys, a, c_hi, c_lo);
    case 6: return launch_l<6>(L, n, n_polys, a, c_hi, c_lo);
    case 7: return launch_l<7>(L, n, n_polys, a, c_hi, c_lo);
    case 8: return launch_l<8>(L, n, n_polys, a, c_hi, c_lo);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ elevation
namespace {

constexpr int kElThreads = 256;

// One block per polynomial: the tensor in shared memory (upper and lower, two
// buffers each), one pass per variable, a thread per line of a pass.
__global__ void __launch_bounds__(kElThreads)
k_bern_elevate(int n, int l, int r, int64_t n_polys, const float* __restrict__ a_hi,
               const float* __restrict__ a_lo, float* __restrict__ c_hi,
               float* __restrict__ c_lo, int go_max, int* status) {
  extern __shared__ float se[];
  __shared__ float2 s_rcp[kMaxEncloseOrder + 1];   // [RD, RU] of 1 / C(l + r, k)
  float* bh[2] = {se, se + go_max};
  float* bl[2] = {se + 2 * go_max, se + 3 * go_max};
  const int Ri = l + 1, Ro = l + r + 1;
  for (int k = threadIdx.x; k < Ro; k += kElThreads)
    s_rcp[k] = make_float2(__frcp_rd(binomf(l + r, k)), __frcp_ru(binomf(l + r, k)));
  int Gi = 1, Go = 1;
  for (int k = 0; k < n; ++k) {
    Gi *= Ri;
    Go *= Ro;
  }
  for (int64_t p = blockIdx.x; p < n_polys; p += gridDim.x) {
    __syncthreads();   // (the first time: s_rcp)
    for (int g = threadIdx.x; g < Gi; g += kElThreads) {
      bh[0][g] = a_hi[p * Gi + g];
      bl[0][g] = a_lo[p * Gi + g];
    }
    __syncthreads();
    int cur = 0;
    // before pass k: variables < k at order l + r, the others at order l
    for (int k = 0; k < n; ++k) {
      int stride = 1;   // of variable k (the last variable is the fastest)
      for (int q = k + 1; q < n; ++q) stride *= Ri;
      int gk = stride * Ro;
      for (int q = 0; q < k; ++q) gk *= Ro;
      const float* ih = bh[cur];
      const float* il = bl[cur];
      float* oh = bh[cur ^ 1];
      float* ol = bl[cur ^ 1];
      // a thread per line (the cells that differ only in variable k)
      const int nl = gk / Ro;
      for (int line = threadIdx.x; line < nl; line += kElThreads) {
        const int inner = line % stride, outer = line / stride;
        const float* xh = ih + outer * (Ri * stride) + inner;
        const float* xl = il + outer * (Ri * stride) + inner;
        float* yh = oh + outer * (Ro * stride) + inner;
        float* yl = ol + outer * (Ro * stride) + inner;
        for (int kk = 0; kk < Ro; ++kk) {
          float hu = 0.0f, hl = 0.0f;
          const int j0 = max(0, kk - r), j1 = min(l, kk);
          for (int j = j0; j <= j1; ++j) {
            const float wl = binomf(l, j), wr = binomf(r, kk - j);
            hu = __fmaf_ru(__fmul_ru(xh[j * stride], wl), wr, hu);
            hl = __fmaf_rd(__fmul_rd(xl[j * stride], wl), wr, hl);
          }
          // x / C with a bracket [q_lo, q_hi] of 1/C: the end that moves x * q
          // up (down) is picked by the sign of x
          const float2 q = s_rcp[kk];
          yh[kk * stride] = __fmul_ru(hu, hu >= 0.0f ? q.y : q.x);
          yl[kk * stride] = __fmul_rd(hl, hl >= 0.0f ? q.x : q.y);
        }
      }
      __syncthreads();
      cur ^= 1;
    }
    for (int g = threadIdx.x; g < Go; g += kElThreads) {
      const float vh = bh[cur][g], vl = bl[cur][g];
      c_hi[p * Go + g] = vh;
      c_lo[p * Go + g] = vl;
      if (!isfinite(vh) || !isfinite(vl)) atomicOr(status, kStatusNonFinite);
    }
    __syncthreads();   // the buffers are reused by the next polynomial
  }
}

__global__ void k_fill_i32(int32_t* __restrict__ x, int64_t count, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// The bias on coefficients 1 .. G-1 of every output neuron (coefficient 0
// got it in the affine step), upward for the upper and downward for the lower
// tensor.
__global__ void k_bias_rows(int64_t n_boxes, int h, int G, const float* __restrict__ bias,
                            float* __restrict__ out_hi, float* __restrict__ out_lo) {
  const int64_t total = n_boxes * (int64_t)(G - 1) * h;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(i % h);
    const int64_t rest = i / h;
    const int64_t g = 1 + rest % (G - 1), b = rest / (G - 1);
    const int64_t o = (b * G + g) * h + m;
    out_hi[o] = __fadd_ru(out_hi[o], bias[m]);
    out_lo[o] = __fadd_rd(out_lo[o], bias[m]);
  }
}

}  // namespace

size_t bernstein_elevate_smem(int n, int l, int r) {
  if (n < 1 || n > kMaxVars || l < 0 || r < 0 || l + r > kMaxEncloseOrder) return SIZE_MAX;
  int64_t go = 1;
  for (int k = 0; k < n; ++k) {
    go *= l + r + 1;
    if (go > (1 << 20)) return SIZE_MAX;
  }
  return (size_t)4 * go * sizeof(float);
}

cudaError_t launch_bernstein_elevate(const Launch& L, int n, int l, int r, int64_t n_polys,
                                     const float* a_hi, const float* a_lo, float* c_hi,
                                     float* c_lo) {
  if (n_polys == 0) return cudaSuccess;
  const size_t smem = bernstein_elevate_smem(n, l, r);
  if (n_polys < 0 || smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bern_elevate,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int go = (int)(smem / (4 * sizeof(float)));
  const int per_sm = std::max(1, std::min(8, (int)((228 * 1024) / (smem + 1024))));
  const int64_t blocks = std::min<int64_t>(n_polys, (int64_t)device_sms(L) * per_sm);
  k_bern_elevate<<<(unsigned)blocks, kElThreads, smem, L.stream>>>(n, l, r, n_polys, a_hi, a_lo,
                                                                   c_hi, c_lo, go, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_bernstein_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                                    const float* W, const float* b, int G, const float* in_hi,
                                    const float* in_lo, float* out_hi, float* out_lo,
                                    int32_t* nt_scratch) {
  if (n_boxes == 0) return cudaSuccess;
  if (n_boxes < 0 || G < 1 || !nt_scratch) return cudaErrorInvalidValue;
  const int64_t nin = n_boxes * h_in;   // input counts first, output counts after them
  const unsigned fb = (unsigned)std::min<int64_t>((nin + 255) / 256, device_sms(L) * 8);
  k_fill_i32<<<fb, 256, 0, L.stream>>>(nt_scratch, nin, G);
  ++*L.launches;
  cudaError_t e = launch_affine(L, n_boxes, h_out, h_in, W, b, in_hi, in_lo, G, nt_scratch,
                                out_hi, out_lo, G, nt_scratch + nin);
  if (e != cudaSuccess || G == 1) return e;
  const int64_t total = n_boxes * (int64_t)(G - 1) * h_out;
  const unsigned bb = (unsigned)std::min<int64_t>((total + 255) / 256, device_sms(L) * 8);
  k_bias_rows<<<bb, 256, 0, L.stream>>>(n_boxes, h_out, G, b, out_hi, out_lo);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
