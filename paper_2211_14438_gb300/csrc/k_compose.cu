// a4: Step 3 of Sec. 5.1 (eqs. post_bounds_1/2): compose the ReLU
// polynomial with the neuron's pre-activation bounds,
//
//   post_up(t) = B(s_up(t)),   post_lo(t) = B(s_lo(t)) - eps,
//   s(t) = (pre(t) - lo) / (hi - lo)  in [0,1] on the box,
//
// as polynomials in t over the graded monomial order, truncated at the
// total-degree cap (dropped terms enter the constant as [min(0,c),max(0,c)]).
//
// Rounding.  s~ = fl((pre - lo*[K=0]) * fl(1/(hi-lo))) is formed in
// round-to-nearest; eta = 5u * sum|s~_K| bounds |s~(t) - s(t)| on the box,
// and Lip = sum_j j|a_j|(1+eta)^(j-1) bounds |B'| there, so Lip*eta is added
// to the upper constant and subtracted from the lower one.  The polynomial
// B(s~(t)) itself is then formed with outward rounding:
//   d = 1: c_K = a0[K=0] + a1 s~_K                  (one directed FMA)
//   d = 2: c_K = a0[K=0] + a1 s~_K + a2 (s~^2)_K     (a2 >= 0 by convexity)
//          with (s~^2)_K = sum_{I+J=K} s~_I s~_J over the symmetric pair list,
//          accumulated round-up for the upper bound, round-down for the lower.
//   d >= 3: Horner q <- q s~ + a_j with interval coefficients [q_lo, q_hi]
//          (both ends accumulated outward, the end used chosen by the sign
//          of s~_J), truncated at the cap after every product with the
//          dropped mass carried as a one-sided remainder through later
//          products by s in [-eta, 1+eta].
//
// One block per (box, neuron) item; threads stride over output monomials;
// the normalised input polynomials live in shared memory.
#include "device_util.cuh"

namespace bern {

constexpr float kU = 0x1p-24f;   // unit roundoff of float32

__device__ __forceinline__ int degree_of(const Tables& T, int m) {
  int D = 0;
  while (D < kMaxTableDegree && T.mcount[D] < m) ++D;
  return D;
}

__global__ void __launch_bounds__(256)
k_compose(Tables T, int cap, float tau, const int8_t* __restrict__ kind,
          const float* __restrict__ coef, const float* __restrict__ eps,
          const uint8_t* __restrict__ degrees, int global_d, const float* __restrict__ lo,
          const float* __restrict__ hi, const float* __restrict__ pre_up,
          const float* __restrict__ pre_lo, int64_t pre_stride,
          const int32_t* __restrict__ pre_nterms, float* __restrict__ post_up,
          float* __restrict__ post_lo, int64_t post_stride, int32_t* __restrict__ post_nterms,
          int* status) {
  extern __shared__ float smem[];
  __shared__ float red[32];
  __shared__ float c0[2];
  const int64_t item = blockIdx.x;
  const int k = kind[item];
  const int Mpre = pre_nterms[item];
  const float* Pu = pre_up + item * pre_stride;
  const float* Pl = pre_lo + item * pre_stride;
  float* Qu = post_up + item * post_stride;
  float* Ql = post_lo + item * post_stride;
  if (k == 0) {
    if (threadIdx.x == 0) post_nterms[item] = 0;
    return;
  }
  if (Mpre > pre_stride || Mpre < 0) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusInvalid);
      post_nterms[item] = 0;
    }
    return;
  }
  if (k == 1) {
    if (Mpre > post_stride) {
      if (threadIdx.x == 0) {
        atomicOr(status, kStatusCapacity);
        post_nterms[item] = 0;
      }
      return;
    }
    for (int r = threadIdx.x; r < Mpre; r += blockDim.x) {
      Qu[r] = Pu[r];
      Ql[r] = Pl[r];
    }
    if (threadIdx.x == 0) post_nterms[item] = Mpre;
    return;
  }
  const int d = degrees ? (int)degrees[item] : global_d;
  const int Dpre = degree_of(T, Mpre);
  // the input is read as the full graded prefix of its degree (missing
  // entries are zero), which must fit the caller's stride
  const int Mp = T.mcount[Dpre];
  if (Mp > pre_stride || d < 1) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusInvalid);
      post_nterms[item] = 0;
    }
    return;
  }
  const int Dfull = d * Dpre;
  const int Dout = min(Dfull, cap);
  if (Dfull > kMaxTableDegree || (d == 2 && Dpre > T.dmax) || d > 2 || tau > 0.0f) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusUnsupported);
      post_nterms[item] = 0;
    }
    return;
  }
  const int Mout = T.mcount[Dout];
  const int Mfull = T.mcount[Dfull];
  if (Mout > post_stride) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusCapacity);
      post_nterms[item] = 0;
    }
    return;
  }
  const float L = lo[item], H = hi[item];
  const float inv = 1.0f / (H - L);
  float* su = smem;
  float* sl = smem + pre_stride;
  float au = 0.0f, al = 0.0f;
  for (int r = threadIdx.x; r < Mp; r += blockDim.x) {
    float vu = r < Mpre ? Pu[r] : 0.0f, vl = r < Mpre ? Pl[r] : 0.0f;
    if (r == 0) {
      vu = __fsub_rn(vu, L);
      vl = __fsub_rn(vl, L);
    }
    vu = __fmul_rn(vu, inv);
    vl = __fmul_rn(vl, inv);
    su[r] = vu;
    sl[r] = vl;
    au = __fadd_ru(au, fabsf(vu));
    al = __fadd_ru(al, fabsf(vl));
  }
  au = block_dsum<true>(au, red);
  __syncthreads();
  al = block_dsum<true>(al, red);
  const float eta_u = __fmul_ru(5.0f * kU, au);
  const float eta_l = __fmul_ru(5.0f * kU, al);
  float a[3];
  const float* cf = coef + item * kCoefStride;
  for (int j = 0; j <= d; ++j) a[j] = cf[j];
  // Lipschitz bound of B on [-eta, 1+eta]
  auto lip = [&](float eta) {
    float s = 0.0f, p = 1.0f;
    for (int j = 1; j <= d; ++j) {
      s = __fmaf_ru((float)j * fabsf(a[j]), p, s);
      p = __fmul_ru(p, __fadd_ru(1.0f, eta));
    }
    return s;
  };
  float remU = 0.0f, remL = 0.0f;
  if (d == 1) {
    for (int K = threadIdx.x; K < Mp; K += blockDim.x) {
      float cu = __fmaf_ru(a[1], su[K], K == 0 ? a[0] : 0.0f);
      float cl = __fmaf_rd(a[1], sl[K], K == 0 ? a[0] : 0.0f);
      if (K == 0) {
        c0[0] = cu;
        c0[1] = cl;
      } else {
        Qu[K] = cu;
        Ql[K] = cl;
      }
    }
  } else {  // d == 2
    const PairTable pt = T.sq[Dpre];
    const bool a2pos = a[2] >= 0.0f;
    for (int K = threadIdx.x; K < Mfull; K += blockDim.x) {
      const int p0 = pt.ptr[K], p1 = pt.ptr[K + 1];
      float offU = 0.0f, offL = 0.0f, diagU = 0.0f, diagL = 0.0f;
      for (int p = p0; p < p1; ++p) {
        const uint32_t pr = pt.pairs[p];
        const int i = pr & 0xffff, j = pr >> 16;
        if (i == j) {
          diagU = __fmul_ru(su[i], su[i]);
          diagL = __fmul_rd(sl[i], sl[i]);
        } else {
          offU = __fmaf_ru(su[i], su[j], offU);
          offL = __fmaf_rd(sl[i], sl[j], offL);
        }
      }
      // (s^2)_K = diag + 2*off  (2*x is exact)
      const float sqU = __fadd_ru(diagU, 2.0f * offU);
      const float sqL = __fadd_rd(diagL, 2.0f * offL);
      // lower bound of a2*(s^2)_K: a2 >= 0 uses the lower end, else the upper
      const float cu = __fmaf_ru(a[2], a2pos ? sqU : sqL,
                                 __fmaf_ru(a[1], K < Mp ? su[K] : 0.0f, K == 0 ? a[0] : 0.0f));
      const float cl = __fmaf_rd(a[2], a2pos ? sqL : sqU,
                                 __fmaf_rd(a[1], K < Mp ? sl[K] : 0.0f, K == 0 ? a[0] : 0.0f));
      if (K == 0) {
        c0[0] = cu;
        c0[1] = cl;
      } else if (K < Mout) {
        Qu[K] = cu;
        Ql[K] = cl;
      } else {
        remU = __fadd_ru(remU, fmaxf(cu, 0.0f));
        remL = __fadd_rd(remL, fminf(cl, 0.0f));
      }
    }
  }
  __syncthreads();
  remU = block_dsum<true>(remU, red);
  __syncthreads();
  remL = block_dsum<false>(remL, red);
  if (threadIdx.x == 0) {
    const float e = eps[item];
    float cu = __fadd_ru(c0[0], __fmul_ru(lip(eta_u), eta_u));
    cu = __fadd_ru(cu, remU);
    float cl = __fsub_rd(c0[1], __fmul_ru(lip(eta_l), eta_l));
    cl = __fsub_rd(cl, e);
    cl = __fadd_rd(cl, remL);
    Qu[0] = cu;
    Ql[0] = cl;
    post_nterms[item] = Mout;
    if (!isfinite(cu) || !isfinite(cl)) atomicOr(status, kStatusNonFinite);
  }
}

cudaError_t launch_compose(const Launch& L, const Tables& T, int64_t n_items, int cap,
                           float tau, const int8_t* kind, const float* coef,
                           const float* eps, const uint8_t* degrees, int global_d,
                           const float* lo, const float* hi, const float* pre_up,
                           const float* pre_lo, int64_t pre_stride,
                           const int32_t* pre_nterms, float* post_up, float* post_lo,
                           int64_t post_stride, int32_t* post_nterms) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = 2 * (size_t)pre_stride * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_compose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_compose<<<(unsigned)n_items, 256, smem, L.stream>>>(
      T, cap, tau, kind, coef, eps, degrees, global_d, lo, hi, pre_up, pre_lo, pre_stride,
      pre_nterms, post_up, post_lo, post_stride, post_nterms, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
