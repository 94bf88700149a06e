// Lin linearisation (Sec. 5.3): every Lin hidden layers the post-activation
// bounds are lowered to order [1,...,1], i.e. to multilinear polynomials.  The
// cited algorithm is not given; the reading here: A is the least-squares
// multilinear fit of the bound P on the box (minimising the integral of
// (P - A)^2 over [0,1]^n), the residual P - A is enclosed by its Bernstein
// coefficients at the layer's order (Def. 2), and the bound becomes A plus the
// residual's maximum (upper bound) or minimum (lower bound).
//
// The fit in closed form: the products prod_{k in S} (2 t_k - 1) over the
// variable sets S (shifted Legendre polynomials of degree 0 or 1 in each
// variable) are orthogonal on [0,1]^n with squared norm 3^-|S|, so
//   A   = sum_S c_S prod_{k in S} (2 t_k - 1),
//   c_S = 3^|S| sum_K p_K prod_{k in S} e_k / ((e_k+1)(e_k+2)) prod_{k not in S} 1/(e_k+1)
// (the integrals of t^K times the basis function), and in the power basis
//   a_T = 2^|T| sum_{S contains T} (-1)^(|S|-|T|) c_S.
// c_S is exactly 0 unless some term contains every variable of S (a factor
// e_k = 0 in its weight vanishes otherwise), so the fit of a degree-D
// polynomial has degree <= min(n, D).
//
// Soundness does not depend on the fit: A enters the bound exactly as stored
// (float32).  The residual coefficients are rounded up (upper) or down
// (lower); every monomial is >= 0 on the box, so the rounded residual bounds
// the exact one pointwise; the enclosure rounds outward; the shift is added
// to A's constant with a directed add.
//
// Layer-block layout as everywhere: coefficient r of neuron m of box b at
// ((b*ld + r)*h + m); nterms[b*h + m] is a graded prefix length (0: the zero
// polynomial).
#include <algorithm>

#include "device_util.cuh"

namespace bern {

namespace {

constexpr int kLinItemsPerBlock = 4;      // two warps (upper, lower) per item
constexpr int kLinMaxSets = 1 << kMaxVars;

// One warp per (item, bound).  Writes the fit A (graded ranks < ntl, zero at
// non-multilinear ranks) to lin and the rounded residual over P in place.
__global__ void __launch_bounds__(64 * kLinItemsPerBlock)
k_lin_project(Tables T, int64_t n_items, int h, int64_t mlin, float* __restrict__ post_up,
              float* __restrict__ post_lo, int64_t ld, const int32_t* __restrict__ nterms,
              float* __restrict__ lin_up, float* __restrict__ lin_lo, int64_t lin_ld,
              int32_t* __restrict__ lin_nt, int* status) {
  __shared__ float s_c[2 * kLinItemsPerBlock][kLinMaxSets];
  __shared__ float s_a[2 * kLinItemsPerBlock][kLinMaxSets];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * kLinItemsPerBlock + (warp >> 1);
  if (item >= n_items) return;            // warp-uniform; no block barrier below
  const bool up = warp & 1;
  const int n = T.n;
  const int NS = 1 << n;
  int nt = nterms[item];
  if (nt < 0 || nt > ld || nt > T.mexps) {
    if (lane == 0) atomicOr(status, kStatusInvalid);
    nt = 0;
  }
  const int ntl = nt < mlin ? nt : (int)mlin;
  const int64_t b = item / h, m = item - b * h;
  float* P = (up ? post_up : post_lo) + (b * ld) * h + m;
  float* A = (up ? lin_up : lin_lo) + (b * lin_ld) * h + m;
  float* sc = s_c[warp];
  float* sa = s_a[warp];
  // c_S, one warp-wide sum per variable set (fixed tree: deterministic)
  for (int S = 0; S < NS; ++S) {
    float acc = 0.0f;
    for (int r = lane; r < nt; r += 32) {
      const uint8_t* e = T.exps + (int64_t)r * n;
      float w = P[(int64_t)r * h];
      for (int k = 0; k < n; ++k) {
        const float ek = (float)e[k];
        w *= ((S >> k) & 1) ? ek / ((ek + 1.0f) * (ek + 2.0f)) : 1.0f / (ek + 1.0f);
      }
      acc += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      float s3 = 1.0f;
      for (int k = 0; k < n; ++k)
        if ((S >> k) & 1) s3 *= 3.0f;
      sc[S] = acc * s3;
    }
  }
  __syncwarp();
  // power-basis coefficients a_T from the supersets S of T
  for (int Tm = lane; Tm < NS; Tm += 32) {
    const int comp = (NS - 1) & ~Tm;
    float a = 0.0f;
    for (int sub = comp;; sub = (sub - 1) & comp) {
      const float c = sc[Tm | sub];
      a += (__popc(sub) & 1) ? -c : c;
      if (sub == 0) break;
    }
    sa[Tm] = a * (float)(1 << __popc(Tm));
  }
  __syncwarp();
  for (int r = lane; r < nt; r += 32) {
    const uint8_t* e = T.exps + (int64_t)r * n;
    bool ml = true;
    int mask = 0;
    for (int k = 0; k < n; ++k) {
      if (e[k] > 1) ml = false;
      else if (e[k] == 1) mask |= 1 << k;
    }
    const float a = ml ? sa[mask] : 0.0f;
    if (ml) {
      const float p = P[(int64_t)r * h];
      P[(int64_t)r * h] = up ? __fsub_ru(p, a) : __fsub_rd(p, a);
    }
    if (r < ntl) A[(int64_t)r * h] = a;
  }
  if (up && lane == 0) lin_nt[item] = ntl;
}

// A's constant += the residual's enclosure (upper: max, rounded up; lower:
// min, rounded down).  Items with no terms stay the zero polynomial.
__global__ void k_lin_shift(int64_t n_items, int h, const int32_t* __restrict__ lin_nt,
                            const float* __restrict__ rlo, const float* __restrict__ rhi,
                            float* __restrict__ lin_up, float* __restrict__ lin_lo,
                            int64_t lin_ld, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items || lin_nt[i] <= 0) return;
  const int64_t b = i / h, m = i - b * h;
  const int64_t o = (b * lin_ld) * h + m;
  const float u = __fadd_ru(lin_up[o], rhi[i]);
  const float l = __fadd_rd(lin_lo[o], rlo[i]);
  lin_up[o] = u;
  lin_lo[o] = l;
  if (!(isfinite(u) && isfinite(l))) atomicOr(status, kStatusNonFinite);
}

}  // namespace

cudaError_t launch_linearize(const Launch& L, const Tables& T, int64_t n_boxes, int h, int order,
                             int64_t budget, float* post_up, float* post_lo, int64_t ld,
                             const int32_t* nterms, float* lin_up, float* lin_lo, int64_t lin_ld,
                             int32_t* lin_nt, float* rlo, float* rhi) {
  const int64_t n_items = n_boxes * h;
  if (n_items == 0) return cudaSuccess;
  const int64_t mlin = num_monomials(T.n, std::min(T.n, order));
  if (T.n > kMaxVars || mlin < 1 || lin_ld < mlin) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((n_items + kLinItemsPerBlock - 1) / kLinItemsPerBlock);
  k_lin_project<<<blocks, 64 * kLinItemsPerBlock, 0, L.stream>>>(
      T, n_items, h, mlin, post_up, post_lo, ld, nterms, lin_up, lin_lo, lin_ld, lin_nt,
      L.status);
  ++*L.launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the residuals (same term counts as the bounds) enclosed at the layer's order
  e = launch_enclose(L, T, n_boxes, h, order, budget, post_up, post_lo, ld, nterms, rlo, rhi);
  if (e != cudaSuccess) return e;
  k_lin_shift<<<(unsigned)((n_items + 255) / 256), 256, 0, L.stream>>>(
      n_items, h, lin_nt, rlo, rhi, lin_up, lin_lo, lin_ld, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
