// a4 for ReLU orders d >= 3, and for every order when pruning is on: Step 3
// of Sec. 5.1 by Horner's rule on polynomials in t,
//
//   q <- a_d;   q <- q * s~ + a_j   (j = d-1, ..., 0),
//
// truncating q at the total-degree cap after every product and, with
// pruning, dropping the terms with |c| < tau * ||q||_1.  Every dropped term
// c t^K lies in [min(0,c), max(0,c)] on the box.
//
// Rounding.  s~ is formed in round-to-nearest as in the order-2 kernels, so
// s~(t) lies within eta = 5u*sum|s~_K| of s(t) in [0,1], i.e. in
// [-eta, 1+eta].  q carries interval coefficients [q_lo, q_up] and an
// interval remainder rho(t) in [R_lo, R_up] (R_lo <= 0 <= R_up) for the
// dropped part:
//   product coefficients   sum over pairs of q_I s~_J with the end of q_I
//                          picked by the sign of s~_J, round-up for the
//                          upper end and round-down for the lower end;
//   carried remainder      rho * s~ in [R_lo(1+eta) - R_up eta,
//                                       R_up(1+eta) - R_lo eta];
//   dropped terms          R_up += max(0, c_up), R_lo += min(0, c_lo).
// The upper bound polynomial is q_up + R_up + Lip*eta (from s~ of the upper
// pre-activation polynomial), the lower one q_lo + R_lo - Lip*eta - eps
// (from s~ of the lower one), with Lip = sum_j j|a_j|(1+eta)^(j-1) bounding
// |B'| on [-eta, 1+eta].
//
// Precision.  Orders below kHornerF64Order run in float32 (u = 2^-24) on the
// coefficients of the enclosure step.  From that order on, the power-form
// coefficients a_j reach C(d, d/2) 2^(d/2) (hi - lo) / d (about 1e5 (hi - lo)
// at d = 16) while q ends of the order of hi - lo, so the float32 roundings
// of the intermediate q would dominate the bound; those items run the same
// steps in float64 (u = 2^-53, directed float64 FMAs), with a_j and eps
// recomputed in float64 from [lo, hi], and every output coefficient is
// rounded outward to float32 (up for the upper polynomial, down for the
// lower one; the monomials are >= 0 on the box, so this moves each
// polynomial outward).
//
// Work layout.  One block of 256 threads per (item, bound): s~ and the two
// ends of q (current and next) sit in shared memory; threads take output
// monomials K of a product and walk the host-built pair list of K (I + J = K).
// Polynomials too large for shared memory keep the same buffers in a slice
// of a global workspace per block (same arithmetic, same order).
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "compose_common.cuh"
#include "relu_form.cuh"

namespace bern {

namespace {

constexpr int kHornerThreads = 256;

// Directed arithmetic in the kernel's precision.
template <typename R>
struct Dir;
template <>
struct Dir<float> {
  static constexpr float u = 0x1p-24f;
  static __device__ __forceinline__ float fma_ru(float a, float b, float c) { return __fmaf_ru(a, b, c); }
  static __device__ __forceinline__ float fma_rd(float a, float b, float c) { return __fmaf_rd(a, b, c); }
  static __device__ __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
  static __device__ __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
  static __device__ __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
  static __device__ __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
  static __device__ __forceinline__ float mul_rd(float a, float b) { return __fmul_rd(a, b); }
  static __device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float out_ru(float a) { return a; }
  static __device__ __forceinline__ float out_rd(float a) { return a; }
};
template <>
struct Dir<double> {
  static constexpr double u = 0x1p-53;
  static __device__ __forceinline__ double fma_ru(double a, double b, double c) { return __fma_ru(a, b, c); }
  static __device__ __forceinline__ double fma_rd(double a, double b, double c) { return __fma_rd(a, b, c); }
  static __device__ __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
  static __device__ __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
  static __device__ __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }
  static __device__ __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }
  static __device__ __forceinline__ double mul_rd(double a, double b) { return __dmul_rd(a, b); }
  static __device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
  // the float32 output of an upper (lower) coefficient: rounded up (down)
  static __device__ __forceinline__ float out_ru(double a) { return __double2float_ru(a); }
  static __device__ __forceinline__ float out_rd(double a) { return __double2float_rd(a); }
};

// Block-wide directed sum in the kernel's precision (every thread gets it).
template <bool UP, typename R>
__device__ R block_dsum_r(R v, R* scratch) {
  if constexpr (std::is_same<R, float>::value) {
    return block_dsum<UP>(v, scratch);
  } else {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, v, o);
      v = UP ? __dadd_ru(v, x) : __dadd_rd(v, x);
    }
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, r, o);
      r = UP ? __dadd_ru(r, x) : __dadd_rd(r, x);
    }
    return r;
  }
}

// sum_j j |a_j| (1+eta)^(j-1), rounded up
template <typename R>
__device__ R horner_lip(const R* a, int d, R eta) {
  using O = Dir<R>;
  R lip = 0, pw = 1;
  const R g = O::add_ru(R(1), eta);
  for (int j = 1; j <= d; ++j) {
    lip = O::fma_ru((R)j * fabs(a[j]), pw, lip);
    pw = O::mul_ru(pw, g);
  }
  return lip;
}

// R = float: queue kQHorner, the ReLU coefficients and shift of the
// enclosure step (float32).  R = double: queue kQHorner64, the coefficients
// and shift recomputed here in float64 from the item's [lo, hi] (the same
// polynomial, without the float32 rounding of its coefficients).
template <typename R>
__global__ void __launch_bounds__(kHornerThreads)
k_compose_horner(Tables T, ComposeArgs A, ComposeScratch S, int ms_cap, int mq_cap,
                 float* gws, int64_t gstride, int* status) {
  using O = Dir<R>;
  constexpr bool kF64 = std::is_same<R, double>::value;
  constexpr int kQ = kF64 ? kQHorner64 : kQHorner;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the buffers: shared memory, or this block's slice of the global workspace
  R* smem = gws ? reinterpret_cast<R*>(gws + (int64_t)blockIdx.x * gstride)
                : reinterpret_cast<R*>(smem_raw);
  __shared__ R red[32];
  __shared__ R s_a[kMaxOrder + 2];   // float64 variant: coefficients and the shift
  __shared__ int s_nz;
  const int tid = threadIdx.x;
  const int count = S.qcount[kQ];
  const int h = A.h;
  for (int task = blockIdx.x; task < 2 * count; task += gridDim.x) {
    const bool up = task & 1;
    const int64_t item = S.queue[(int64_t)kQ * S.qcap + (task >> 1)];
    const int Mpre = A.pre_nterms[item];
    const int D = degree_of(T, Mpre);
    const int Ms = T.mcount[D];
    const int d = A.degrees ? (int)A.degrees[item] : A.global_d;
    // shapes the launcher sized the buffers for (checked again here)
    const int Dfin = min(d * D, A.cap);
    if (Ms > ms_cap || T.mcount[Dfin] > mq_cap || d < 1 || d > kMaxOrder) {
      if (tid == 0) atomicOr(status, kStatusUnsupported);
      continue;
    }
    R* s = smem;
    R* qu = s + ms_cap;
    R* ql = qu + mq_cap;
    R* nu = ql + mq_cap;
    R* nl = nu + mq_cap;
    const R Lo = A.lo[item], Hi = A.hi[item];
    const R inv = R(1) / (Hi - Lo);
    const float* P = (up ? A.pre_up : A.pre_lo) + A.base(item, A.pre_ld);
    if constexpr (kF64) {
      if (tid == 0) relu_power_form_t<double>(A.lo[item], A.hi[item], d, s_a, s_a + kMaxOrder + 1);
    }
    R l1 = 0;
    for (int r = tid; r < Ms; r += kHornerThreads) {
      R v = r < Mpre ? (R)P[(int64_t)r * h] : R(0);
      if (r == 0) v = O::sub_rn(v, Lo);
      v = O::mul_rn(v, inv);
      s[r] = v;
      l1 = O::add_ru(l1, fabs(v));
    }
    l1 = block_dsum_r<true>(l1, red);   // (its barriers also publish s_a)
    const R eta = O::mul_ru(R(5) * O::u, l1);
    const R g = O::add_ru(R(1), eta);
    R a[kMaxOrder + 1];
    R eps_item;
    if constexpr (kF64) {
#pragma unroll
      for (int j = 0; j <= kMaxOrder; ++j) a[j] = j <= d ? s_a[j] : 0.0;
      eps_item = s_a[kMaxOrder + 1];
    } else {
      const float* cf = A.coef + item * kCoefStride;
#pragma unroll
      for (int j = 0; j <= kMaxOrder; ++j) a[j] = j <= d ? cf[j] : 0.0f;
      eps_item = A.eps[item];
    }
    if (tid == 0) {
      qu[0] = a[d];
      ql[0] = a[d];
    }
    __syncthreads();
    int Dq = 0;
    R Rup = 0, Rlo = 0;   // identical in every thread
    bool ok = true;
    for (int j = d - 1; j >= 0; --j) {
      const int Dp = Dq + D, Dk = min(Dp, A.cap);
      const ProdTable pt = T.prod[Dq * kProdStride + D];
      if (Dp > kMaxTableDegree || pt.ptr == nullptr) {
        if (tid == 0) atomicOr(status, kStatusUnsupported);
        ok = false;
        break;
      }
      const int Mp = T.mcount[Dp], Mk = T.mcount[Dk];
      // carried remainder rho * s~ (R_lo <= 0 <= R_up)
      const R cRup = O::fma_ru(-Rlo, eta, O::mul_ru(Rup, g));
      const R cRlo = O::fma_rd(-Rup, eta, O::mul_rd(Rlo, g));
      R dru = 0, drl = 0;
      for (int K = tid; K < Mp; K += kHornerThreads) {
        const int p0 = __ldg(pt.ptr + K), p1 = __ldg(pt.ptr + K + 1);
        R cu = K == 0 ? a[j] : R(0), cl = cu;
        for (int p = p0; p < p1; ++p) {
          const int2 pr = __ldg(pt.pairs + p);
          const R sv = s[pr.y];
          const R xu = qu[pr.x], xl = ql[pr.x];
          const bool pos = sv >= R(0);
          cu = O::fma_ru(pos ? xu : xl, sv, cu);
          cl = O::fma_rd(pos ? xl : xu, sv, cl);
        }
        if (K < Mk) {
          nu[K] = cu;
          nl[K] = cl;
        } else {
          dru = O::add_ru(dru, fmax(cu, R(0)));
          drl = O::add_rd(drl, fmin(cl, R(0)));
        }
      }
      dru = block_dsum_r<true>(dru, red);
      drl = block_dsum_r<false>(drl, red);
      Rup = O::add_ru(cRup, dru);
      Rlo = O::add_rd(cRlo, drl);
      if (A.tau > 0.0f) {
        // pruning (relative to the L1 norm of this bound's end of q)
        R nrm = 0;
        for (int K = tid; K < Mk; K += kHornerThreads) nrm = O::add_ru(nrm, fabs(up ? nu[K] : nl[K]));
        nrm = block_dsum_r<true>(nrm, red);
        const R thr = (R)A.tau * nrm;
        R pru = 0, prl = 0;
        for (int K = 1 + tid; K < Mk; K += kHornerThreads) {
          if (fabs(up ? nu[K] : nl[K]) < thr) {
            pru = O::add_ru(pru, fmax(nu[K], R(0)));
            prl = O::add_rd(prl, fmin(nl[K], R(0)));
            nu[K] = 0;
            nl[K] = 0;
          }
        }
        pru = block_dsum_r<true>(pru, red);
        prl = block_dsum_r<false>(prl, red);
        Rup = O::add_ru(Rup, pru);
        Rlo = O::add_rd(Rlo, prl);
      }
      __syncthreads();
      R* t0 = qu;
      qu = nu;
      nu = t0;
      t0 = ql;
      ql = nl;
      nl = t0;
      Dq = Dk;
    }
    if (!ok) continue;
    const int Mout = T.mcount[Dq];
    float* Q = (up ? A.post_up : A.post_lo) + A.base(item, A.post_ld);
    if (tid == 0) s_nz = 1;
    __syncthreads();
    int nz = 1;
    for (int K = 1 + tid; K < Mout; K += kHornerThreads) {
      const float v = up ? O::out_ru(qu[K]) : O::out_rd(ql[K]);
      Q[(int64_t)K * h] = v;
      if (v != 0.0f) nz = K + 1;
    }
    if (A.tau > 0.0f) {
      nz = warp_imax(nz);
      if ((tid & 31) == 0) atomicMax(&s_nz, nz);
    }
    __syncthreads();
    if (tid == 0) {
      const R lip = horner_lip(a, d, eta);
      const R le = O::mul_ru(lip, eta);
      float v;
      if (up) {
        v = O::out_ru(O::add_ru(O::add_ru(qu[0], Rup), le));
      } else {
        R w = O::sub_rd(O::add_rd(ql[0], Rlo), le);
        v = O::out_rd(O::sub_rd(w, eps_item));
      }
      Q[0] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
      // with pruning, the term count is the graded prefix up to the highest
      // degree with a kept term (both bounds share it)
      if (A.tau > 0.0f) atomicMax(&A.post_nterms[item], T.mcount[degree_of(T, s_nz)]);
    }
    __syncthreads();
  }
}

}  // namespace

namespace {

// Buffer floats per block of one variant (s~ and four ends of q, in float or
// double elements), SIZE_MAX when a size is out of range.
size_t variant_floats(const Tables& T, int Dmax, int Dout, bool f64) {
  const int64_t ms = num_monomials(T.n, Dmax), mq = num_monomials(T.n, Dout);
  if (ms < 0 || mq < 0) return SIZE_MAX;
  return ((size_t)ms + 4 * (size_t)mq) * (f64 ? 2 : 1);
}

// Output degrees of the two variants for inputs of degree <= Dmax and orders
// <= d: float32 items have orders below kHornerF64Order (or any order <= 2
// with pruning), float64 items the rest.
int dout_f32(int Dmax, int cap, int d) {
  return std::min(cap, std::max(1, std::min(d, kHornerF64Order - 1)) * Dmax);
}
int dout_f64(int Dmax, int cap, int d) { return std::min(cap, d * Dmax); }

bool in_global(size_t floats, int64_t smem_limit) {
  return (int64_t)(floats * sizeof(float)) > std::min<int64_t>(smem_limit, 200 * 1024);
}

template <typename R>
cudaError_t launch_variant(const Launch& L, const Tables& T, const ComposeScratch& S,
                           const ComposeArgs& A, int Dmax, int Dout) {
  constexpr bool kF64 = std::is_same<R, double>::value;
  const size_t floats = variant_floats(T, Dmax, Dout, kF64);
  if (floats == SIZE_MAX) return cudaErrorInvalidValue;
  const int ms_cap = (int)num_monomials(T.n, Dmax), mq_cap = (int)num_monomials(T.n, Dout);
  if (in_global(floats, S.horner_smem_limit)) {
    if (!S.hws || S.hws_blocks < 1 || S.hws_floats < (int64_t)(floats * S.hws_blocks))
      return cudaErrorInvalidValue;
    k_compose_horner<R><<<S.hws_blocks, kHornerThreads, 0, L.stream>>>(
        T, A, S, ms_cap, mq_cap, S.hws, (int64_t)floats, L.status);
    ++*L.launches;
    return cudaGetLastError();
  }
  const size_t smem = floats * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_compose_horner<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int per_sm = std::max(1, std::min(8, (int)((228 * 1024) / (smem + 1024))));
  k_compose_horner<R><<<device_sms(L) * per_sm, kHornerThreads, smem, L.stream>>>(
      T, A, S, ms_cap, mq_cap, nullptr, 0, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace

size_t horner_smem_floats(const Tables& T, int Dmax, int cap, int d) {
  size_t f = variant_floats(T, Dmax, dout_f32(Dmax, cap, d), false);
  if (d >= kHornerF64Order && f != SIZE_MAX)
    f = std::max(f, variant_floats(T, Dmax, dout_f64(Dmax, cap, d), true));
  return f;
}

size_t horner_global_floats(const Tables& T, int Dmax, int cap, int d, int64_t smem_limit,
                            int blocks) {
  size_t need = 0;
  const size_t f32 = variant_floats(T, Dmax, dout_f32(Dmax, cap, d), false);
  if (f32 == SIZE_MAX) return SIZE_MAX;
  if (in_global(f32, smem_limit)) need = f32 * (size_t)blocks;
  if (d >= kHornerF64Order) {
    const size_t f64 = variant_floats(T, Dmax, dout_f64(Dmax, cap, d), true);
    if (f64 == SIZE_MAX) return SIZE_MAX;
    if (in_global(f64, smem_limit)) need = std::max(need, f64 * (size_t)blocks);
  }
  return need;
}

cudaError_t launch_compose_horner(const Launch& L, const Tables& T, const ComposeScratch& S,
                                  const ComposeArgs& A, int Dmax) {
  const int d = std::max(1, A.global_d);
  const bool f64 = d >= kHornerF64Order;
  // float32 items exist unless every item has order d >= kHornerF64Order
  if ((A.tau > 0.0f || d >= 3) && (A.degrees != nullptr || !f64)) {
    cudaError_t e = launch_variant<float>(L, T, S, A, Dmax, dout_f32(Dmax, A.cap, d));
    if (e != cudaSuccess) return e;
  }
  if (f64) return launch_variant<double>(L, T, S, A, Dmax, dout_f64(Dmax, A.cap, d));
  return cudaSuccess;
}

}  // namespace bern
