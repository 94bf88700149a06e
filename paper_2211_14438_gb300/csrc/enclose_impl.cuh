// a2: Step 1 of Sec. 5.1 (eq. find_lo_hi) via the range enclosing property
// (Def. 2):  lo = min_I b_I(pre_lo),  hi = max_I b_I(pre_up),
// where b_I are the coefficients of the exact Bernstein expansion of order l
// (in every variable) on [0,1]^n of a power-form polynomial a_J:
//
//   b_I = sum_{J <= I} prod_k C(i_k, j_k) / C(l, j_k) * a_J.
//
// After scaling c_J = a_J / prod_k C(l, j_k), the map factors into one
// transform per variable, c -> (sum_{j<=i} C(i,j) c_j)_i, whose weights are
// exact small integers.  The scaling multiplies by a float bracket of the
// reciprocal (the end chosen by the sign of a_J and the rounding direction),
// and the transforms use directed FMAs (round-down for the lower polynomial,
// round-up for the upper one), so every computed coefficient is a one-sided
// bound of the exact one.
//
// Work layout.  One warp per polynomial; a block holds 2*P warps = P items
// (warp 2i: lower polynomial of item i, warp 2i+1: upper).  Each warp stages
// the (l+1)^n grid in shared memory, indexed in mixed radix (l+1) with t_1 the
// slowest digit; host-built tables per order give each graded rank's grid
// index and each line's base offset and prefix digit sum, so the kernels do
// no mixed-radix arithmetic.  A polynomial of total degree D <= l occupies only the
// simplex sum_k j_k <= D, so the transforms run from the last variable to the
// first, each over the lines whose untransformed prefix still lies in the
// simplex, reading only in-simplex inputs (no zero fill needed).  A line is
// loaded into registers, transformed with compile-time binomial weights and
// written back; the first variable's transform feeds the min/max directly.
//
// a3 (fused): once both bounds of an item are known, one thread computes the
// ReLU case and the order-d Bernstein polynomial of ReLU on [lo, hi]
// (Def. 1, Prop. 1) in the power basis of s = (y-lo)/(hi-lo), plus the shift
// B(0) of Prop. 2 (eq. max_error), in float64 rounded up to float32 with a
// margin that covers the float64 error.
#pragma once
#include <math_constants.h>

#include <algorithm>
#include <string>

#include "device_util.cuh"
#include "relu_form.cuh"

namespace bern {

constexpr int kEncloseGridMax = BERN_MAX_GRID;   // floats per warp (96 KB)

constexpr float cbin(int i, int j) {
  float r = 1.0f;
  for (int k = 1; k <= j; ++k) r = r * (float)(i - j + k) / (float)k;
  return r;
}


// ------------------------------------------------------------------ a2
// In place, from the top: y_i needs x_0 .. x_i only, so x_i can take y_i
// once it is formed (same FMAs in the same order as line_transform).
template <int LB, bool UP>
__device__ __forceinline__ void line_transform_inplace(float (&x)[LB + 1]) {
#pragma unroll
  for (int i = LB; i >= 1; --i) {
    float acc = x[0];
#pragma unroll
    for (int j = 1; j <= i; ++j) acc = dfma<UP>(cbin(i, j), x[j], acc);
    x[i] = acc;
  }
}

template <int LB, bool UP>
__device__ __forceinline__ void line_transform(const float (&x)[LB + 1], float (&y)[LB + 1]) {
#pragma unroll
  for (int i = 0; i <= LB; ++i) {
    float acc = x[0];
#pragma unroll
    for (int j = 1; j <= i; ++j) acc = dfma<UP>(cbin(i, j), x[j], acc);
    y[i] = acc;
  }
}

// Scatter the scaled coefficients of the first m_eff graded ranks (degree
// <= Deff) into the grid at their precomputed grid indices; return the
// directed sum of the one-sided ranges of all other terms.  Coefficient r is
// P[r * ps], or P[pos[r]] when PERM (a polynomial held in another order, e.g.
// the row layout of the fused layer kernel).
template <bool UP, bool PERM = false>
__device__ float scatter_terms(const float* __restrict__ P, int ps, int nt,
                               const int32_t* __restrict__ gidx, const float2* __restrict__ rs,
                               int m_eff, float* grid, const int32_t* __restrict__ pos = nullptr) {
  const int lane = threadIdx.x & 31;
  float rem = 0.0f;
  for (int r = lane; r < nt; r += 32) {
    const float a = PERM ? P[__ldg(pos + r)] : P[(int64_t)r * ps];
    if (r < m_eff) {
      const float2 sc = rs[r];
      // a / C bracketed: choose the end that rounds the product the right way
      grid[__ldg(gidx + r)] = UP ? __fmul_ru(a, a >= 0.0f ? sc.y : sc.x)
                                 : __fmul_rd(a, a >= 0.0f ? sc.x : sc.y);
    } else {
      // the term lies in [min(0,a), max(0,a)] on the box
      rem = UP ? __fadd_ru(rem, fmaxf(a, 0.0f)) : __fadd_rd(rem, fminf(a, 0.0f));
    }
  }
  // a ragged count (not a full graded prefix): missing simplex entries are 0
  for (int r = nt + lane; r < m_eff; r += 32) grid[__ldg(gidx + r)] = 0.0f;
  return rem;
}

// R^e for small e
__device__ __forceinline__ int ipow(int R, int e) {
  int p = 1;
  for (int i = 0; i < e; ++i) p *= R;
  return p;
}
constexpr int cipow(int R, int e) { return e == 0 ? 1 : R * cipow(R, e - 1); }

// Lines of pass k whose prefix digit sum is <= D: C(D + k, k) prefixes times
// R^(n-1-k) suffixes, for D <= R-1.  From four variables on the line tables
// put those of D = R-1 first in each pass, so a loop over that many lines
// (skipping prefix sums above the polynomial's degree) covers every line the
// polynomial needs; below, the loops cover all lines.
__device__ __forceinline__ int simplex_lines(int D, int k, int suffixes) {
  if (D + k > kMaxEncloseOrder) {   // beyond the exact binomial table
    int c = 1;
    for (int i = 1; i <= k; ++i) c = c * (D + i) / i;
    return c * suffixes;
  }
  return (int)binomf(D + k, k) * suffixes;   // C(D + k, k), exact in float
}

// Total degree of a graded prefix of nt terms (the smallest D with M(n,D) >= nt).
__device__ __forceinline__ int prefix_degree(const Tables& T, int nt) {
  return nt <= T.mexps ? (int)T.deg_of[nt] : kMaxTableDegree;
}

// One pass of the warp enclosure: the lines along variable k (prefix digits,
// variables < k, untransformed; suffix digits, variables > k, transformed),
// sk the stride of variable k, nl the lines looped over, nlines the lines of
// a pass in the table.  The last pass (k == 0) takes the extreme into best.
// NV == 3: the line's base and prefix sum follow from Ln (the line tables'
// order: the low digit of Ln is the highest variable other than k) instead of
// a table load.
template <int LB, bool UP, int NV = 0>
__device__ __forceinline__ void enclose_pass(int k, int sk, int nl, int nlines,
                                             const int2* __restrict__ lines, int Deff,
                                             float* grid, float& best) {
  constexpr int R = LB + 1;
  const int lane = threadIdx.x & 31;
  for (int Ln = lane; Ln < nl; Ln += 32) {
    int base, psum;
    if constexpr (NV == 3) {
      const int q = Ln / R, r = Ln - q * R;
      base = k == 2 ? Ln * R : k == 1 ? q * (R * R) + r : Ln;
      psum = k == 2 ? q + r : k == 1 ? q : 0;
    } else {
      const int2 ln = __ldg(lines + (int64_t)k * nlines + Ln);
      base = ln.x;
      psum = ln.y;
    }
    if (psum > Deff) continue;
    const int p = Deff - psum;
    float x[R], y[R];
#pragma unroll
    for (int j = 0; j < R; ++j) x[j] = j <= p ? grid[base + j * sk] : 0.0f;
    // in place up to order 8 (fewer live registers); above, the separate
    // output array schedules better (measured)
    if constexpr (LB <= 8) {
      line_transform_inplace<LB, UP>(x);
#pragma unroll
      for (int i = 0; i < R; ++i) y[i] = x[i];
    } else {
      line_transform<LB, UP>(x, y);
    }
    if (k > 0) {
#pragma unroll
      for (int i = 0; i < R; ++i) grid[base + i * sk] = y[i];
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) best = UP ? fmaxf(best, y[i]) : fminf(best, y[i]);
    }
  }
}

// SIMP: loop over the in-simplex prefix of each pass (tables of four or more
// variables, see simplex_lines); otherwise over all lines.  NV > 0: the
// variable count is NV at compile time (n == NV), so the passes unroll and
// the line strides become immediate offsets.
template <int LB, bool UP, bool PERM = false, bool SIMP = false, int NV = 0>
__device__ float enclose_warp(const float* __restrict__ P, int ps, int nt, int n,
                              const Tables& T, const float2* __restrict__ rs, float* grid,
                              const int32_t* __restrict__ pos = nullptr) {
  static_assert(NV == 0 || NV == 3, "compiled variable counts");
  constexpr int R = LB + 1;
  const int Dnt = prefix_degree(T, nt);
  const int Deff = Dnt < LB ? Dnt : LB;
  float rem = scatter_terms<UP, PERM>(P, ps, nt, T.gidx[LB], rs, T.mcount[Deff], grid, pos);
  __syncwarp();
  float best = UP ? -CUDART_INF_F : CUDART_INF_F;
  const int2* __restrict__ lines = T.lines[LB];
  if constexpr (NV > 0) {
    constexpr int nlines = cipow(R, NV - 1);
#pragma unroll
    for (int k = NV - 1; k >= 0; --k) {
      const int sk = cipow(R, NV - 1 - k);
      enclose_pass<LB, UP, NV>(k, sk, nlines, nlines, lines, Deff, grid, best);
      __syncwarp();
    }
  } else {
    const int nlines = ipow(R, n - 1);
    for (int k = n - 1; k >= 0; --k) {
      const int sk = ipow(R, n - 1 - k);
      const int nl = SIMP ? simplex_lines(LB, k, sk) : nlines;
      enclose_pass<LB, UP>(k, sk, nl, nlines, lines, Deff, grid, best);
      __syncwarp();
    }
  }
  best = UP ? warp_max(best) : warp_min(best);
  rem = warp_dsum<UP>(rem);
  return dadd<UP>(best, rem);
}

// Options of one enclosure launch: the fused a3 outputs (kind == nullptr:
// enclosure only) and an optional item list (list != nullptr: the launch
// covers items list[0 .. *count), a device-side count; otherwise items
// 0 .. n_items).
struct EncloseOpts {
  int8_t* kind;
  float* coef;
  float* eps;
  const uint8_t* degrees;
  int global_d;
  const int* list = nullptr;
  const int* count = nullptr;
};

__device__ __forceinline__ int64_t map_item(const EncloseOpts& o, int64_t idx, int64_t n_items) {
  if (o.list) return idx < *o.count ? (int64_t)o.list[idx] : -1;
  return idx < n_items ? idx : -1;
}

// Orders up to 6 fit 32 registers without spills: four 512-thread blocks per
// SM (64 warps); higher orders keep three.
// SIMP as in enclose_warp; NV > 0: compiled for NV variables
template <int LB, bool SIMP, int NV>
__global__ void __launch_bounds__(512, (LB <= 6 ? 4 : 3))
k_enclose(Tables T, int G, const float2* __restrict__ rs, int64_t n_items, int h,
          const float* __restrict__ pre_up, const float* __restrict__ pre_lo, int64_t ld,
          const int32_t* __restrict__ nterms, float* __restrict__ lo, float* __restrict__ hi,
          EncloseOpts ro, int* status) {
  extern __shared__ float smem[];
  __shared__ float s_lohi[8][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_block = blockDim.x >> 6;               // items per block
  const int64_t item = map_item(ro, (int64_t)blockIdx.x * per_block + (warp >> 1), n_items);
  const bool up = warp & 1;
  if (item >= 0) {
    int nt = nterms[item];
    if (nt < 0 || nt > ld || nt > T.mexps) {
      if (lane == 0) atomicOr(status, kStatusInvalid);
      nt = 0;
    }
    const int64_t b = item / h;
    const int64_t base = (b * ld) * h + (item - b * h);
    float* grid = smem + warp * G;
    const float v =
        up ? enclose_warp<LB, true, false, SIMP, NV>(pre_up + base, h, nt, T.n, T, rs, grid)
           : enclose_warp<LB, false, false, SIMP, NV>(pre_lo + base, h, nt, T.n, T, rs, grid);
    if (lane == 0) {
      (up ? hi : lo)[item] = v;
      s_lohi[warp >> 1][up ? 1 : 0] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  }
  if (ro.kind == nullptr) return;
  __syncthreads();
  if (threadIdx.x < per_block) {
    const int64_t it = map_item(ro, (int64_t)blockIdx.x * per_block + threadIdx.x, n_items);
    if (it >= 0) {
      const int d = ro.degrees ? (int)ro.degrees[it] : ro.global_d;
      ro.kind[it] = (int8_t)relu_item(s_lohi[threadIdx.x][0], s_lohi[threadIdx.x][1], d,
                                      ro.coef + it * kCoefStride, ro.eps + it, status);
    }
  }
}

template <int LB>
cudaError_t launch_lb(const Launch& L, const Tables& T, int G, int64_t n_items, int h,
                      const float* pre_up, const float* pre_lo, int64_t ld,
                      const int32_t* nterms, float* lo, float* hi, EncloseOpts ro) {
  // items per block: as many as fit 192 KB of grids, at most 8 (16 warps);
  // autotuned among 8, 4 and 2 (variants 0, 1, 2; variants 3 and 4, a block
  // per polynomial, are taken before this launcher where they apply, and run
  // as variant 2 where they do not)
  int items = (int)std::min<int64_t>(8, (192 * 1024) / (2 * (int64_t)G * 4));
  const std::string key = "enclose/" + std::to_string(LB) + "/" + std::to_string(T.n) + "/" +
                          std::to_string(n_items);
  const int v = tune_variant(L, "enclose", key, 0);
  items = std::min(items, 8 >> std::min(v, 2));
  if (items < 1) items = 1;
  TuneTimer tt;
  tune_begin(L, "enclose", tt);
  const size_t smem = (size_t)2 * items * G * sizeof(float);
  // the in-simplex prefix loop for four or more variables (their grids of
  // l >= 12, 13^4 cells and more, exceed kEncloseGridMax and run elsewhere)
  auto kern = k_enclose<LB, false, 0>;
  if constexpr (LB >= 4)   // three-variable grids of l <= 3 take the small-grid kernel
    if (T.n == 3) kern = k_enclose<LB, false, 3>;
  if constexpr (LB <= 11)
    if (T.n >= 4) kern = k_enclose<LB, true, 0>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((n_items + items - 1) / items);
  kern<<<blocks, 64 * items, smem, L.stream>>>(T, G, T.rscale[LB], n_items, h, pre_up, pre_lo,
                                               ld, nterms, lo, hi, ro, L.status);
  ++*L.launches;
  const cudaError_t e = cudaGetLastError();
  tune_end(L, "enclose", key, tt);
  return e;
}

// Tiny grids ((l+1)^n <= 64): one lane per polynomial, the lane's grid
// interleaved with its warp's (element g of lane L at grid[g*32 + L]); a warp
// takes 32 items of one bound, a block 4 groups of 32 items (both bounds).
constexpr int kSmallGrid = 64;
template <int LB, bool UP>
__device__ float enclose_lane(const float* __restrict__ P, int ps, int nt, int n,
                              const Tables& T, const float2* __restrict__ rs, float* grid) {
  constexpr int R = LB + 1;
  const int32_t* __restrict__ gidx = T.gidx[LB];
  const int2* __restrict__ lines = T.lines[LB];
  const int Dnt = prefix_degree(T, nt);
  const int Deff = Dnt < LB ? Dnt : LB;
  const int m_eff = T.mcount[Deff];
  float rem = 0.0f;
  for (int r = 0; r < nt; ++r) {
    const float a = P[(int64_t)r * ps];
    if (r < m_eff) {
      const float2 sc = rs[r];
      grid[__ldg(gidx + r) * 32] = UP ? __fmul_ru(a, a >= 0.0f ? sc.y : sc.x)
                                      : __fmul_rd(a, a >= 0.0f ? sc.x : sc.y);
    } else {
      rem = UP ? __fadd_ru(rem, fmaxf(a, 0.0f)) : __fadd_rd(rem, fminf(a, 0.0f));
    }
  }
  for (int r = nt; r < m_eff; ++r) grid[__ldg(gidx + r) * 32] = 0.0f;
  float best = UP ? -CUDART_INF_F : CUDART_INF_F;
  const int nlines = ipow(R, n - 1);
  for (int k = n - 1; k >= 0; --k) {
    const int sk = ipow(R, n - 1 - k);
    const int nl = n >= 4 ? simplex_lines(LB, k, sk) : nlines;
    for (int Ln = 0; Ln < nl; ++Ln) {
      const int2 ln = __ldg(lines + (int64_t)k * nlines + Ln);
      const int base = ln.x, psum = ln.y;
      if (psum > Deff) continue;
      const int p = Deff - psum;
      float x[R], y[R];
#pragma unroll
      for (int j = 0; j < R; ++j) x[j] = j <= p ? grid[(base + j * sk) * 32] : 0.0f;
      line_transform<LB, UP>(x, y);
      if (k > 0) {
#pragma unroll
        for (int i = 0; i < R; ++i) grid[(base + i * sk) * 32] = y[i];
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) best = UP ? fmaxf(best, y[i]) : fminf(best, y[i]);
      }
    }
  }
  return dadd<UP>(best, rem);
}

template <int LB>
__global__ void __launch_bounds__(256)
k_enclose_small(Tables T, int G, const float2* __restrict__ rs, int64_t n_items, int h,
                const float* __restrict__ pre_up, const float* __restrict__ pre_lo, int64_t ld,
                const int32_t* __restrict__ nterms, float* __restrict__ lo,
                float* __restrict__ hi, EncloseOpts ro, int* status) {
  extern __shared__ float smem[];
  __shared__ float s_lohi[128][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = warp >> 1;
  const bool up = warp & 1;
  const int64_t item = map_item(ro, (int64_t)blockIdx.x * 128 + group * 32 + lane, n_items);
  float v = 0.0f;
  if (item >= 0) {
    int nt = nterms[item];
    if (nt < 0 || nt > ld || nt > T.mexps) {
      atomicOr(status, kStatusInvalid);
      nt = 0;
    }
    const int64_t b = item / h;
    const int64_t base = (b * ld) * h + (item - b * h);
    float* grid = smem + (size_t)warp * G * 32 + lane;
    v = up ? enclose_lane<LB, true>(pre_up + base, h, nt, T.n, T, rs, grid)
           : enclose_lane<LB, false>(pre_lo + base, h, nt, T.n, T, rs, grid);
    (up ? hi : lo)[item] = v;
    if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
  }
  s_lohi[group * 32 + lane][up ? 1 : 0] = v;
  if (ro.kind == nullptr) return;
  __syncthreads();
  if (threadIdx.x < 128) {
    const int64_t it = map_item(ro, (int64_t)blockIdx.x * 128 + threadIdx.x, n_items);
    if (it >= 0) {
      const int d = ro.degrees ? (int)ro.degrees[it] : ro.global_d;
      ro.kind[it] = (int8_t)relu_item(s_lohi[threadIdx.x][0], s_lohi[threadIdx.x][1], d,
                                      ro.coef + it * kCoefStride, ro.eps + it, status);
    }
  }
}

template <int LB>
cudaError_t launch_small(const Launch& L, const Tables& T, int G, int64_t n_items, int h,
                         const float* pre_up, const float* pre_lo, int64_t ld,
                         const int32_t* nterms, float* lo, float* hi, EncloseOpts ro) {
  const size_t smem = (size_t)8 * G * 32 * sizeof(float);   // <= 64 KB
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_enclose_small<LB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((n_items + 127) / 128);
  k_enclose_small<LB><<<blocks, 256, smem, L.stream>>>(T, G, T.rscale[LB], n_items, h, pre_up,
                                                       pre_lo, ld, nterms, lo, hi, ro,
                                                       L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// Orders above 16: one kernel with a runtime order; each line is transformed
// in place in shared memory by l sweeps of pairwise directed additions
// (Pascal's rule: after sweep r, c_i holds sum_j C(.,.) c_j partial sums), so
// only non-negative integer weights are applied.
template <bool UP>
__device__ float enclose_warp_generic(const float* __restrict__ P, int ps, int nt, int n,
                                      int lb, const Tables& T, const float2* __restrict__ rs,
                                      float* grid) {
  const int lane = threadIdx.x & 31;
  const int R = lb + 1;
  const int Dnt = prefix_degree(T, nt);
  const int Deff = Dnt < lb ? Dnt : lb;
  float rem = scatter_terms<UP>(P, ps, nt, T.gidx[lb], rs, T.mcount[Deff], grid);
  __syncwarp();
  float best = UP ? -CUDART_INF_F : CUDART_INF_F;
  const int nlines = ipow(R, n - 1);
  const int2* __restrict__ lines = T.lines[lb];
  for (int k = n - 1; k >= 0; --k) {
    const int sk = ipow(R, n - 1 - k);
    const int nl = n >= 4 ? simplex_lines(lb, k, sk) : nlines;
    for (int Ln = lane; Ln < nl; Ln += 32) {
      const int2 ln = __ldg(lines + (int64_t)k * nlines + Ln);
      const int base = ln.x, psum = ln.y;
      if (psum > Deff) continue;
      const int p = Deff - psum;
      float* c = grid + base;
      for (int j = p + 1; j <= lb; ++j) c[j * sk] = 0.0f;
      for (int r = 1; r <= lb; ++r)
        for (int i = lb; i >= r; --i) c[i * sk] = dadd<UP>(c[i * sk], c[(i - 1) * sk]);
      if (k == 0)
        for (int i = 0; i <= lb; ++i) best = UP ? fmaxf(best, c[i * sk]) : fminf(best, c[i * sk]);
    }
    __syncwarp();
  }
  best = UP ? warp_max(best) : warp_min(best);
  rem = warp_dsum<UP>(rem);
  return dadd<UP>(best, rem);
}

}  // namespace bern
