// a3: the order-d Bernstein polynomial of ReLU on [lo, hi] (Def. 1, Prop. 1)
// in the power basis of s = (y - lo)/(hi - lo), and the shift B(0) of Prop. 2
// (eq. max_error) that makes it a sound lower bound once subtracted.
//
// The coefficients are summed in float64 from the samples ReLU(lo + k(hi-lo)/d)
// and rounded up with a margin that covers the float64 error, so each is >=
// the exact coefficient of the Bernstein polynomial of the computed samples;
// the constant coefficient also carries the samples' own rounding (at most
// 5u(hi - lo) when lo < 0 < hi, the only case this is used for), so the
// polynomial is >= the exact Bernstein polynomial on s in [0,1].  The
// returned eps is >= B(s0) (s0 the s of y = 0) plus the sum of every upward
// coefficient excess, so the polynomial minus eps stays below ReLU.  Two
// precisions: float32 coefficients for the float32 composition kernels, and
// float64 ones for the float64 Horner kernel of high orders.  The float32
// path of orders 1 and 2 (the common case) uses their closed forms in float32
// instead (relu_power_form_low): the GPU's float64 units run at a small
// fraction of its float32 rate.
#pragma once

#include <type_traits>

#include "device_util.cuh"

namespace bern {

// C(d,k) for d <= 16, exact in float64
static __constant__ const double c_dbin[17][17] = {
    {1},
    {1, 1},
    {1, 2, 1},
    {1, 3, 3, 1},
    {1, 4, 6, 4, 1},
    {1, 5, 10, 10, 5, 1},
    {1, 6, 15, 20, 15, 6, 1},
    {1, 7, 21, 35, 35, 21, 7, 1},
    {1, 8, 28, 56, 70, 56, 28, 8, 1},
    {1, 9, 36, 84, 126, 126, 84, 36, 9, 1},
    {1, 10, 45, 120, 210, 252, 210, 120, 45, 10, 1},
    {1, 11, 55, 165, 330, 462, 462, 330, 165, 55, 11, 1},
    {1, 12, 66, 220, 495, 792, 924, 792, 495, 220, 66, 12, 1},
    {1, 13, 78, 286, 715, 1287, 1716, 1716, 1287, 715, 286, 78, 13, 1},
    {1, 14, 91, 364, 1001, 2002, 3003, 3432, 3003, 2002, 1001, 364, 91, 14, 1},
    {1, 15, 105, 455, 1365, 3003, 5005, 6435, 6435, 5005, 3003, 1365, 455, 105, 15, 1},
    {1, 16, 120, 560, 1820, 4368, 8008, 11440, 12870, 11440, 8008, 4368, 1820, 560, 120, 16, 1}};

static __device__ __forceinline__ double dbin(int d, int k) { return c_dbin[d][k]; }

// R = float or double: the precision of the returned coefficients and shift
template <typename R>
static __device__ void relu_power_form_t(float lo, float hi, int d, R* a_out, R* eps_out) {
  const double L = lo, H = hi, w = H - L;
  const double inv_d = 1.0 / (double)d;
  double b[kMaxOrder + 1];
  for (int k = 0; k <= d; ++k) {
    double node = L + w * ((double)k * inv_d);   // Def. 1 grid point
    b[k] = node > 0.0 ? node : 0.0;
  }
  double excess = 0.0;
  for (int j = 0; j <= d; ++j) {
    double s = 0.0, mag = 0.0;
    for (int k = 0; k <= j; ++k) {
      // coefficient of s^j in C(d,k) s^k (1-s)^(d-k)
      double t = b[k] * (dbin(d, k) * dbin(d - k, j - k));
      s += ((j - k) & 1) ? -t : t;
      mag += t;
    }
    double margin = mag * 0x1p-40;
    if (j == 0) margin += w * 0x1p-48;   // the samples' rounding (constant term)
    if constexpr (std::is_same<R, float>::value) {
      const float aj = __double2float_ru(s + margin);
      a_out[j] = aj;
      excess += ((double)aj - s) + margin;
    } else {
      const double aj = __dadd_ru(s, margin);
      a_out[j] = aj;
      excess = __dadd_ru(excess, __dadd_ru(__dsub_ru(aj, s), margin));
    }
  }
  const double s0 = -L / w;
  double e = 0.0;
  for (int k = 0; k <= d; ++k) {
    double t = b[k] * dbin(d, k);
    for (int i = 0; i < k; ++i) t *= s0;
    for (int i = 0; i < d - k; ++i) t *= (1.0 - s0);
    e += t;
  }
  if constexpr (std::is_same<R, float>::value)
    *eps_out = __double2float_ru((e + excess) * (1.0 + 0x1p-40) + w * 0x1p-40);
  else
    *eps_out = __dadd_ru(__dmul_ru(__dadd_ru(e, excess), 1.0 + 0x1p-40), w * 0x1p-40);
}

static __device__ __forceinline__ void relu_power_form(float lo, float hi, int d, float* a_out,
                                                       float* eps_out) {
  relu_power_form_t<float>(lo, hi, d, a_out, eps_out);
}

// Orders 1 and 2 in closed form, float32 with directed rounding (lo < 0 < hi,
// w = hi - lo, s0 = -lo / w).  Order 1: B(s) = hi s (the chord), B(s0) =
// -lo hi / w.  Order 2: the middle sample is max((lo + hi)/2, 0); when lo + hi
// > 0, B(s) = (lo + hi) s - lo s^2 and B(s0) = -lo hi^2 / w^2, otherwise
// B(s) = hi s^2 and B(s0) = hi lo^2 / w^2 (the sign of the float sum lo + hi
// is that of the exact one).  Every coefficient is exact but lo + hi, which
// is rounded up; its excess and the shift are bounded with upward roundings of
// positive quantities (w rounded down where it divides).
static __device__ void relu_power_form_low(float lo, float hi, int d, float* a_out,
                                           float* eps_out) {
  const float wd = __fsub_rd(hi, lo);
  float a1, a2 = 0.0f, excess = 0.0f, e;
  if (d == 1) {
    a1 = hi;
    e = __fdiv_ru(__fmul_ru(-lo, hi), wd);
  } else if (__fadd_rn(lo, hi) > 0.0f) {
    a1 = __fadd_ru(lo, hi);
    a2 = -lo;
    excess = __fsub_ru(a1, __fadd_rd(lo, hi));   // >= a1 - (lo + hi)
    e = __fdiv_ru(__fmul_ru(-lo, __fmul_ru(hi, hi)), __fmul_rd(wd, wd));
  } else {
    a1 = 0.0f;
    a2 = hi;
    e = __fdiv_ru(__fmul_ru(hi, __fmul_ru(lo, lo)), __fmul_rd(wd, wd));
  }
  a_out[0] = 0.0f;
  a_out[1] = a1;
  if (d == 2) a_out[2] = a2;
  *eps_out = __fadd_ru(e, excess);
}

// Case of one item and, for case 2, its coefficients.  Returns the case.
static __device__ int relu_item(float l, float h, int d, float* a, float* eps, int* status) {
  if (!(isfinite(l) && isfinite(h))) {
    atomicOr(status, kStatusNonFinite);
    return 0;
  }
  if (h <= 0.0f) return 0;        // ReLU is 0 on [lo,hi]
  if (l >= 0.0f) return 1;        // ReLU is the identity on [lo,hi]
  if (d < 1 || d > kMaxOrder) {
    atomicOr(status, kStatusInvalid);
    return 0;
  }
  if (d <= 2)
    relu_power_form_low(l, h, d, a, eps);
  else
    relu_power_form(l, h, d, a, eps);
  return 2;
}

}  // namespace bern
