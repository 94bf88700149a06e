// Change of variables of the output polynomials from the normalised box
// coordinates back to the input coordinates.  The inputs enter the network as
// x_i = dlo_i + w_i t_i on the box (Sec. 5.3; w_i = dhi_i - dlo_i rounded up,
// as bern_init_inputs forms it), so with a_i = 1 / w_i and b_i = -dlo_i / w_i
//
//   P(t) = sum_K c_K t^K = sum_J e_J x^J,
//   e_J  = sum_{K >= J} c_K prod_i C(k_i, j_i) a_i^{j_i} b_i^{k_i - j_i}
//
// (binomial theorem per variable; a side with w_i = 0 is the point x_i = dlo_i,
// t_i = 0, and keeps only the terms with k_i = 0).
//
// Rounding.  e_J is accumulated in float64 together with E_J, the sum of the
// magnitudes of its terms.  Every table entry C(k,j) a^j b^(k-j) carries a
// relative error below (4D + 2) u (u = 2^-53: the iterated binomial, pow of
// the float64 reciprocal and ratio, two products), a term adds n + 1
// roundings and the sum one per term, so |e_J - e*_J| <= gamma E_J with
// gamma = 2 (n (4D + 3) + nt + 4) u
// (the factor 2 covers the second-order terms).  Each e_J (J != 0) is rounded
// to float to nearest; |float(e_J) - e*_J| <= |float(e_J) - e_J| + gamma E_J =
// err_J, and on the box |x^J| <= X^J with X_i = max(|dlo_i|, |dhi_i|).  The
// constant term takes R = sum_{J != 0} err_J X^J + gamma E_0 (with a relative
// margin for the float64 evaluation of R): c'_0 = RU(e_0 + R) for an upper
// polynomial and RD(e_0 - R) for a lower one, so the converted upper (lower)
// polynomial is >= (<=) the original one everywhere on the box.
//
// Work layout: one warp per polynomial, lanes over the output monomials J;
// per J the warp walks the terms K of degree >= |J| in graded order (all
// lanes read the same K: a broadcast) with per-variable tables of
// C(k,j) a^j b^(k-j) and X^j in shared memory.
#include "device_util.cuh"

namespace bern {

constexpr int kPxWarps = 4;

__global__ void __launch_bounds__(32 * kPxWarps)
k_poly_to_x(Tables T, int n, int64_t n_polys, int o, const float* __restrict__ boxes,
            const int32_t* __restrict__ nterms, const float* __restrict__ coef_t, int64_t cap,
            float* __restrict__ coef_x, int D, int* status) {
  extern __shared__ double dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R1 = D + 1;
  double* pw = dsm + (size_t)warp * n * (R1 * R1 + R1);   // pw[i][k][j]
  double* xp = pw + (size_t)n * R1 * R1;                   // xp[i][j] = X_i^j
  const int64_t poly = (int64_t)blockIdx.x * kPxWarps + warp;
  if (poly >= n_polys) return;                              // no block barrier follows
  const bool upper = (poly & 1) == 0;                       // [box][output][upper, lower]
  const int64_t b = (poly >> 1) / o;
  const float* bx = boxes + b * n * 2;
  int nt = nterms[poly];
  if (nt < 0 || nt > cap || nt > T.mexps) {
    if (lane == 0) atomicOr(status, kStatusInvalid);
    return;
  }
  if (nt == 0) return;
  const int Dp = T.deg_of[nt];
  if (Dp > D) {
    if (lane == 0) atomicOr(status, kStatusInvalid);
    return;
  }
  for (int idx = lane; idx < n * R1; idx += 32) {
    const int i = idx / R1, k = idx - i * R1;
    const float dl = bx[2 * i], dh = bx[2 * i + 1];
    if (!(isfinite(dl) && isfinite(dh) && dl <= dh)) atomicOr(status, kStatusInvalid);
    const float w = __fsub_ru(dh, dl);
    const double a = w > 0.0f ? 1.0 / (double)w : 0.0;
    const double bb = w > 0.0f ? -(double)dl / (double)w : 0.0;
    // row k: C(k, j) a^j b^(k-j), j = 0..k (zero above the diagonal); a zero
    // power factor (a point side, or dlo = 0) gives an exact zero
    double* row = pw + ((size_t)i * R1 + k) * R1;
    double c = 1.0;                                         // C(k, j), j = 0 first
    for (int j = 0; j < R1; ++j) {
      double v = 0.0;
      if (j <= k) {
        const double pa = j == 0 ? 1.0 : pow(a, (double)j);
        const double pb = k == j ? 1.0 : (bb == 0.0 ? 0.0 : pow(bb, (double)(k - j)));
        v = (pa == 0.0 || pb == 0.0) ? 0.0 : c * pa * pb;
        c = c * (double)(k - j) / (double)(j + 1);          // C(k, j + 1)
      }
      row[j] = v;
    }
    const double X = fmax(fabs((double)dl), fabs((double)dh));
    xp[(size_t)i * R1 + k] = k == 0 ? 1.0 : pow(X, (double)k);
  }
  __syncwarp();
  const double gamma =
      2.0 * ((double)n * (4.0 * D + 3.0) + (double)nt + 4.0) * 0x1p-53;
  const uint8_t* __restrict__ ex = T.exps;
  const float* C = coef_t + poly * cap;
  float* Xo = coef_x + poly * cap;
  double rsum = 0.0, e0 = 0.0;
  for (int J0 = 0; J0 < nt; J0 += 32) {
    const int J = J0 + lane;
    const bool live = J < nt;
    int jx[kMaxVars];
    for (int i = 0; i < kMaxVars; ++i) jx[i] = (live && i < n) ? ex[(int64_t)J * n + i] : 0;
    // terms of degree >= the chunk's smallest degree (the degree of rank J0)
    const int dmin = T.deg_of[J0 + 1];
    const int kstart = dmin == 0 ? 0 : T.mcount[dmin - 1];
    double e = 0.0, E = 0.0;
    for (int K = kstart; K < nt; ++K) {
      const double cK = (double)C[K];
      bool ge = live && cK != 0.0;
      double wgt = cK;
      for (int i = 0; i < n; ++i) {
        const int kx = ex[(int64_t)K * n + i];
        ge = ge && kx >= jx[i];
        if (ge) wgt *= pw[((size_t)i * R1 + kx) * R1 + jx[i]];
      }
      if (ge) {
        e += wgt;
        E += fabs(wgt);
      }
    }
    if (live) {
      if (J == 0) {
        e0 = e;
        rsum += gamma * E;
      } else {
        const float ef = __double2float_rn(e);
        Xo[J] = ef;
        double xpJ = 1.0;
        for (int i = 0; i < n; ++i) xpJ *= xp[(size_t)i * R1 + jx[i]];
        rsum += (fabs((double)ef - e) + gamma * E) * xpJ;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, off);
  if (lane == 0) {
    // margin for the float64 evaluation of R (sums and products of
    // non-negative terms) and of e_0 -/+ R
    const double R = rsum * (1.0 + ((double)nt + (double)n * D + 16.0) * 0x1p-51);
    double v = upper ? e0 + R : e0 - R;
    v = upper ? v + fabs(v) * 0x1p-50 : v - fabs(v) * 0x1p-50;
    const float c0 = upper ? __double2float_ru(v) : __double2float_rd(v);
    Xo[0] = c0;
    if (!isfinite(c0)) atomicOr(status, kStatusNonFinite);
  }
}

size_t poly_to_x_smem(int n, int D) {
  const size_t R1 = (size_t)D + 1;
  return (size_t)kPxWarps * n * (R1 * R1 + R1) * sizeof(double);
}

cudaError_t launch_poly_to_x(const Launch& L, const Tables& T, int n, int64_t n_boxes, int o,
                             const float* boxes, const int32_t* nterms, const float* coef_t,
                             int64_t cap, float* coef_x, int D) {
  const int64_t n_polys = n_boxes * o * 2;
  if (n_polys == 0) return cudaSuccess;
  const size_t smem = poly_to_x_smem(n, D);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_poly_to_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (n_polys + kPxWarps - 1) / kPxWarps;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  k_poly_to_x<<<(unsigned)blocks, 32 * kPxWarps, smem, L.stream>>>(
      T, n, n_polys, o, boxes, nterms, coef_t, cap, coef_x, D, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
