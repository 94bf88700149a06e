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
// Work layout.  One block of 256 threads per (item, bound): s~ and the two
// ends of q (current and next) sit in shared memory; threads take output
// monomials K of a product and walk the host-built pair list of K (I + J = K).
// Polynomials too large for shared memory keep the same buffers in a slice
// of a global workspace per block (same arithmetic, same order).
#include <stdint.h>

#include <algorithm>

#include "compose_common.cuh"

namespace bern {

namespace {

constexpr int kHornerThreads = 256;

// sum_j j |a_j| (1+eta)^(j-1), rounded up
__device__ float horner_lip(const float* a, int d, float eta) {
  float lip = 0.0f, pw = 1.0f;
  const float g = __fadd_ru(1.0f, eta);
  for (int j = 1; j <= d; ++j) {
    lip = __fmaf_ru((float)j * fabsf(a[j]), pw, lip);
    pw = __fmul_ru(pw, g);
  }
  return lip;
}

__global__ void __launch_bounds__(kHornerThreads)
k_compose_horner(Tables T, ComposeArgs A, ComposeScratch S, int ms_cap, int mq_cap,
                 float* gws, int64_t gstride, int* status) {
  extern __shared__ float smem_dyn[];
  // the buffers: shared memory, or this block's slice of the global workspace
  float* smem = gws ? gws + (int64_t)blockIdx.x * gstride : smem_dyn;
  __shared__ float red[32];
  __shared__ int s_nz;
  const int tid = threadIdx.x;
  const int count = S.qcount[kQHorner];
  const int h = A.h;
  for (int task = blockIdx.x; task < 2 * count; task += gridDim.x) {
    const bool up = task & 1;
    const int64_t item = S.queue[(int64_t)kQHorner * S.qcap + (task >> 1)];
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
    float* s = smem;
    float* qu = s + ms_cap;
    float* ql = qu + mq_cap;
    float* nu = ql + mq_cap;
    float* nl = nu + mq_cap;
    const float Lo = A.lo[item], Hi = A.hi[item];
    const float inv = 1.0f / (Hi - Lo);
    const float* P = (up ? A.pre_up : A.pre_lo) + A.base(item, A.pre_ld);
    float l1 = 0.0f;
    for (int r = tid; r < Ms; r += kHornerThreads) {
      float v = r < Mpre ? P[(int64_t)r * h] : 0.0f;
      if (r == 0) v = __fsub_rn(v, Lo);
      v = __fmul_rn(v, inv);
      s[r] = v;
      l1 = __fadd_ru(l1, fabsf(v));
    }
    l1 = block_dsum<true>(l1, red);
    const float eta = __fmul_ru(5.0f * kU, l1);
    const float g = __fadd_ru(1.0f, eta);
    float a[kMaxOrder + 1];
    const float* cf = A.coef + item * kCoefStride;
#pragma unroll
    for (int j = 0; j <= kMaxOrder; ++j) a[j] = j <= d ? cf[j] : 0.0f;
    if (tid == 0) {
      qu[0] = a[d];
      ql[0] = a[d];
    }
    __syncthreads();
    int Dq = 0;
    float Rup = 0.0f, Rlo = 0.0f;   // identical in every thread
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
      const float cRup = __fmaf_ru(-Rlo, eta, __fmul_ru(Rup, g));
      const float cRlo = __fmaf_rd(-Rup, eta, __fmul_rd(Rlo, g));
      float dru = 0.0f, drl = 0.0f;
      for (int K = tid; K < Mp; K += kHornerThreads) {
        const int p0 = __ldg(pt.ptr + K), p1 = __ldg(pt.ptr + K + 1);
        float cu = K == 0 ? a[j] : 0.0f, cl = cu;
        for (int p = p0; p < p1; ++p) {
          const int2 pr = __ldg(pt.pairs + p);
          const float sv = s[pr.y];
          const float xu = qu[pr.x], xl = ql[pr.x];
          const bool pos = sv >= 0.0f;
          cu = __fmaf_ru(pos ? xu : xl, sv, cu);
          cl = __fmaf_rd(pos ? xl : xu, sv, cl);
        }
        if (K < Mk) {
          nu[K] = cu;
          nl[K] = cl;
        } else {
          dru = __fadd_ru(dru, fmaxf(cu, 0.0f));
          drl = __fadd_rd(drl, fminf(cl, 0.0f));
        }
      }
      dru = block_dsum<true>(dru, red);
      drl = block_dsum<false>(drl, red);
      Rup = __fadd_ru(cRup, dru);
      Rlo = __fadd_rd(cRlo, drl);
      if (A.tau > 0.0f) {
        // pruning (relative to the L1 norm of this bound's end of q)
        float nrm = 0.0f;
        for (int K = tid; K < Mk; K += kHornerThreads) nrm = __fadd_ru(nrm, fabsf(up ? nu[K] : nl[K]));
        nrm = block_dsum<true>(nrm, red);
        const float thr = A.tau * nrm;
        float pru = 0.0f, prl = 0.0f;
        for (int K = 1 + tid; K < Mk; K += kHornerThreads) {
          if (fabsf(up ? nu[K] : nl[K]) < thr) {
            pru = __fadd_ru(pru, fmaxf(nu[K], 0.0f));
            prl = __fadd_rd(prl, fminf(nl[K], 0.0f));
            nu[K] = 0.0f;
            nl[K] = 0.0f;
          }
        }
        pru = block_dsum<true>(pru, red);
        prl = block_dsum<false>(prl, red);
        Rup = __fadd_ru(Rup, pru);
        Rlo = __fadd_rd(Rlo, prl);
      }
      __syncthreads();
      float* t0 = qu;
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
      const float v = up ? qu[K] : ql[K];
      Q[(int64_t)K * h] = v;
      if (v != 0.0f) nz = K + 1;
    }
    if (A.tau > 0.0f) {
      nz = warp_imax(nz);
      if ((tid & 31) == 0) atomicMax(&s_nz, nz);
    }
    __syncthreads();
    if (tid == 0) {
      const float lip = horner_lip(a, d, eta);
      const float le = __fmul_ru(lip, eta);
      float v;
      if (up) {
        v = __fadd_ru(__fadd_ru(qu[0], Rup), le);
      } else {
        v = __fsub_rd(__fadd_rd(ql[0], Rlo), le);
        v = __fsub_rd(v, A.eps[item]);
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

// Buffer floats (per block) the Horner kernel needs for inputs of degree
// <= Dmax and outputs of degree <= Dout; above kHornerSmemLimit bytes the
// buffers live in global memory.
size_t horner_smem_floats(const Tables& T, int Dmax, int Dout) {
  const int64_t ms = num_monomials(T.n, Dmax), mq = num_monomials(T.n, Dout);
  if (ms < 0 || mq < 0) return SIZE_MAX;
  return (size_t)ms + 4 * (size_t)mq;
}

size_t horner_global_floats(const Tables& T, int Dmax, int Dout, int64_t smem_limit, int blocks) {
  const size_t f = horner_smem_floats(T, Dmax, Dout);
  if (f == SIZE_MAX || (int64_t)(f * sizeof(float)) <= smem_limit) return 0;
  return f * (size_t)blocks;
}

cudaError_t launch_compose_horner(const Launch& L, const Tables& T, const ComposeScratch& S,
                                  const ComposeArgs& A, int Dmax, int Dout) {
  const size_t floats = horner_smem_floats(T, Dmax, Dout);
  if (floats == SIZE_MAX) return cudaErrorInvalidValue;
  const int ms_cap = (int)num_monomials(T.n, Dmax), mq_cap = (int)num_monomials(T.n, Dout);
  if ((int64_t)(floats * sizeof(float)) > std::min<int64_t>(S.horner_smem_limit, 200 * 1024)) {
    if (!S.hws || S.hws_blocks < 1 || S.hws_floats < (int64_t)(floats * S.hws_blocks))
      return cudaErrorInvalidValue;
    k_compose_horner<<<S.hws_blocks, kHornerThreads, 0, L.stream>>>(
        T, A, S, ms_cap, mq_cap, S.hws, (int64_t)floats, L.status);
    ++*L.launches;
    return cudaGetLastError();
  }
  const size_t smem = floats * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_compose_horner,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int per_sm = std::max(1, std::min(8, (int)((228 * 1024) / (smem + 1024))));
  k_compose_horner<<<device_sms(L) * per_sm, kHornerThreads, smem, L.stream>>>(T, A, S, ms_cap, mq_cap,
                                                                      nullptr, 0, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
