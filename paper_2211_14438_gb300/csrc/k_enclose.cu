// a2: Step 1 of Sec. 5.1 (eq. find_lo_hi) via the range enclosing property
// (Def. 2):  lo = min_I b_I(pre_lo),  hi = max_I b_I(pre_up),
// where b_I are the coefficients of the exact Bernstein expansion of order l
// (in every variable) on [0,1]^n of a power-form polynomial a_J:
//
//   b_I = sum_{J <= I} prod_k C(i_k, j_k) / C(l, j_k) * a_J.
//
// It factors into n one-dimensional transforms.  Per variable, after scaling
// c_j = a_j / C(l, j), the map c -> (sum_{j<=i} C(i,j) c_j)_i is computed by
// l sweeps of pairwise additions (Pascal's rule), so only additions of
// non-negative weights occur.  The lower polynomial is processed with
// round-down division/addition and the upper one with round-up, which makes
// every computed coefficient a one-sided bound of the exact one.
//
// a3: Step 2 of Sec. 5.1: the order-d Bernstein polynomial of ReLU on
// [lo, hi] (Def. 1, Prop. 1) in the power basis of s = (y-lo)/(hi-lo), and
// the shift B(0) of Prop. 2 (eq. max_error), evaluated in float64 and
// rounded up to float32 with a margin that covers the float64 error.
//
// Layout: one block of two warps per item; warp 0 takes pre_lo (min), warp 1
// pre_up (max); each stages its (l+1)^n grid in shared memory.
#include <math_constants.h>

#include "device_util.cuh"

namespace bern {

constexpr int kEncloseGridMax = BERN_MAX_GRID;   // floats per warp (96 KB)

template <bool UP>
__device__ float enclose_one(const float* __restrict__ P, int nt, int n, int lb, int G,
                             const uint8_t* __restrict__ exps, float* grid) {
  const int lane = threadIdx.x & 31;
  int pw[kMaxVars];
  {
    int p = 1;
    for (int k = n - 1; k >= 0; --k) {
      pw[k] = p;
      p *= (lb + 1);
    }
  }
  for (int g = lane; g < G; g += 32) grid[g] = 0.0f;
  __syncwarp();
  float rem = 0.0f;
  for (int r = lane; r < nt; r += 32) {
    const float a = P[r];
    const uint8_t* e = exps + (int64_t)r * n;
    int deg = 0, idx = 0;
    for (int k = 0; k < n; ++k) {
      deg += e[k];
      idx += e[k] * pw[k];
    }
    if (deg <= lb) {
      float v = a;
      for (int k = 0; k < n; ++k)
        if (e[k]) v = ddiv<UP>(v, binomf(lb, e[k]));
      grid[idx] = v;
    } else {
      // the term lies in [min(0,a), max(0,a)] on the box
      rem = UP ? __fadd_ru(rem, fmaxf(a, 0.0f)) : __fadd_rd(rem, fminf(a, 0.0f));
    }
  }
  __syncwarp();
  const int nlines = G / (lb + 1);
  for (int k = 0; k < n; ++k) {
    const int sk = pw[k];
    for (int L = lane; L < nlines; L += 32) {
      const int hiP = L / sk, loP = L - hiP * sk;
      float* c = grid + hiP * sk * (lb + 1) + loP;
      for (int rr = 1; rr <= lb; ++rr)
        for (int i = lb; i >= rr; --i) c[i * sk] = dadd<UP>(c[i * sk], c[(i - 1) * sk]);
    }
    __syncwarp();
  }
  float best = UP ? -CUDART_INF_F : CUDART_INF_F;
  for (int g = lane; g < G; g += 32) best = UP ? fmaxf(best, grid[g]) : fminf(best, grid[g]);
  best = UP ? warp_max(best) : warp_min(best);
  rem = warp_dsum<UP>(rem);
  return dadd<UP>(best, rem);
}

__global__ void __launch_bounds__(64)
k_enclose(Tables T, int lb, int G, const float* __restrict__ pre_up,
          const float* __restrict__ pre_lo, int64_t stride, const int32_t* __restrict__ nterms,
          float* __restrict__ lo, float* __restrict__ hi, int* status) {
  extern __shared__ float smem[];
  const int64_t item = blockIdx.x;
  const int warp = threadIdx.x >> 5;
  int nt = nterms[item];
  if (nt < 0 || nt > stride || nt > T.mexps) {
    if (threadIdx.x == 0) atomicOr(status, kStatusInvalid);
    nt = 0;
  }
  float* grid = smem + warp * G;
  if (warp == 0) {
    float v = enclose_one<false>(pre_lo + item * stride, nt, T.n, lb, G, T.exps, grid);
    if ((threadIdx.x & 31) == 0) {
      lo[item] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  } else {
    float v = enclose_one<true>(pre_up + item * stride, nt, T.n, lb, G, T.exps, grid);
    if ((threadIdx.x & 31) == 0) {
      hi[item] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  }
}

// Effective Bernstein order: the requested order, lowered until the grid
// fits both the caller's budget and the shared-memory grid limit (and the
// exact-binomial limit).  Terms above it are enclosed by coefficient
// intervals (budget rule).
int effective_order(int n, int order, int64_t budget, int* grid_out) {
  if (budget <= 0) budget = (int64_t)1 << 20;
  int64_t lim = budget < kEncloseGridMax ? budget : kEncloseGridMax;
  int lb = order < kMaxEncloseOrder ? order : kMaxEncloseOrder;
  for (; lb > 0; --lb) {
    int64_t g = 1;
    for (int k = 0; k < n && g <= lim; ++k) g *= (lb + 1);
    if (g <= lim) break;
  }
  int64_t g = 1;
  for (int k = 0; k < n; ++k) g *= (lb + 1);
  *grid_out = (int)g;
  return lb;
}

cudaError_t launch_enclose(const Launch& L, const Tables& T, int64_t n_items, int order,
                           int64_t budget, const float* pre_up, const float* pre_lo,
                           int64_t stride, const int32_t* nterms, float* lo, float* hi) {
  if (n_items == 0) return cudaSuccess;
  int G;
  int lb = effective_order(T.n, order, budget, &G);
  size_t smem = 2 * (size_t)G * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_enclose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_enclose<<<(unsigned)n_items, 64, smem, L.stream>>>(T, lb, G, pre_up, pre_lo, stride, nterms,
                                                      lo, hi, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ a3
// Order-d Bernstein polynomial of ReLU on [lo,hi], power form in s, every
// coefficient rounded up (>= the exact one); eps >= B(0) + sum_j (a~_j - a_j).
__device__ void relu_power_form(float lo, float hi, int d, float* a_out, float* eps_out) {
  const double L = lo, H = hi, w = H - L;
  double b[kMaxOrder + 1];
  for (int k = 0; k <= d; ++k) {
    double node = L + w * (double)k / (double)d;   // Def. 1 grid point
    b[k] = node > 0.0 ? node : 0.0;
  }
  double excess = 0.0;
  for (int j = 0; j <= d; ++j) {
    double s = 0.0, mag = 0.0;
    for (int k = 0; k <= j; ++k) {
      // coefficient of s^j in C(d,k) s^k (1-s)^(d-k)
      double t = b[k] * binomd(d, k) * binomd(d - k, j - k);
      s += ((j - k) & 1) ? -t : t;
      mag += t;
    }
    const double margin = mag * 0x1p-40;
    const float aj = __double2float_ru(s + margin);
    a_out[j] = aj;
    excess += ((double)aj - s) + margin;
  }
  const double s0 = -L / w;
  double e = 0.0;
  for (int k = 0; k <= d; ++k) {
    double t = b[k] * binomd(d, k);
    for (int i = 0; i < k; ++i) t *= s0;
    for (int i = 0; i < d - k; ++i) t *= (1.0 - s0);
    e += t;
  }
  *eps_out = __double2float_ru((e + excess) * (1.0 + 0x1p-40) + w * 0x1p-40);
}

__global__ void k_relu_coeffs(int64_t n_items, const float* __restrict__ lo,
                              const float* __restrict__ hi, const uint8_t* __restrict__ degrees,
                              int global_d, int8_t* __restrict__ kind, float* __restrict__ coef,
                              float* __restrict__ eps, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const float l = lo[i], h = hi[i];
  float* a = coef + i * kCoefStride;
  if (!(isfinite(l) && isfinite(h))) {
    atomicOr(status, kStatusNonFinite);
    kind[i] = 0;
    return;
  }
  if (h <= 0.0f) {            // ReLU is 0 on [lo,hi]
    kind[i] = 0;
    return;
  }
  if (l >= 0.0f) {            // ReLU is the identity on [lo,hi]
    kind[i] = 1;
    return;
  }
  const int d = degrees ? (int)degrees[i] : global_d;
  if (d < 1 || d > kMaxOrder) {
    atomicOr(status, kStatusInvalid);
    kind[i] = 0;
    return;
  }
  kind[i] = 2;
  relu_power_form(l, h, d, a, eps + i);
}

cudaError_t launch_relu_coeffs(const Launch& L, int64_t n_items, const float* lo,
                               const float* hi, const uint8_t* degrees, int global_d,
                               int8_t* kind, float* coef, float* eps) {
  if (n_items == 0) return cudaSuccess;
  k_relu_coeffs<<<(unsigned)((n_items + 127) / 128), 128, 0, L.stream>>>(
      n_items, lo, hi, degrees, global_d, kind, coef, eps, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
