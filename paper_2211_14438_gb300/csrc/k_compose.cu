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
// B(s~(t)) itself is formed with outward rounding:
//   d = 1: c_K = a0[K=0] + a1 s~_K                  (one directed FMA)
//   d = 2: c_K = a0[K=0] + a1 s~_K + a2 (s~^2)_K     (a2 >= 0 by convexity)
// where (s~^2)_K is accumulated round-up for the upper bound and round-down
// for the lower one (a2 >= 0, so each end bounds a2*(s~^2)_K correctly).
//
// Work layout.  A classification kernel puts each item (box, neuron) into a
// queue: zero items only get a term count of 0; identity items and order-1
// items go to an elementwise kernel; order-2 items of input degree D <= 8 go
// to queue D of the row-convolution kernel (one lane per item, 32 items of
// equal structure per warp), the rest to a per-item pair-list kernel.
#include <algorithm>

#include "compose_common.cuh"
#include "row_conv.cuh"

namespace bern {

// ------------------------------------------------------------ classification
// Each block classifies 1024 consecutive items and appends them to the
// queues in item order (ballot/popc within a warp, a scan over the warps),
// reserving its range of every queue with one atomic; so a queue is a list
// of sorted runs, and a warp's 32 consecutive entries are mostly neighbouring
// neurons of one box.
__global__ void __launch_bounds__(1024)
k_compose_queue(Tables T, ComposeArgs A, int64_t n_items, int row_dmax, ComposeScratch S,
                int* status) {
  __shared__ int s_wcnt[32][kComposeQueues];
  __shared__ int s_base[kComposeQueues];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int q = -1;
  if (item < n_items) {
    const int k = A.kind[item];
    const int Mpre = A.pre_nterms[item];
    int nt = 0;
    if (Mpre < 0 || Mpre > A.pre_cap) {
      atomicOr(status, kStatusInvalid);
    } else if (k == 1) {
      if (Mpre > A.post_ld) {
        atomicOr(status, kStatusCapacity);
      } else {
        q = kQIdent;
        nt = Mpre;
      }
    } else if (k == 2) {
      const int d = A.degrees ? (int)A.degrees[item] : A.global_d;
      const int D = degree_of(T, Mpre);
      if (T.mcount[D] > A.pre_cap || d < 1 || d > kMaxOrder || (A.degrees && d > A.global_d)) {
        atomicOr(status, kStatusInvalid);
      } else {
        const int Mout = T.mcount[min(d * D, A.cap)];
        if (Mout > A.post_ld) {
          atomicOr(status, kStatusCapacity);
        } else if (A.tau > 0.0f || d >= 3) {
          q = d >= kHornerF64Order ? kQHorner64 : kQHorner;
          nt = A.tau > 0.0f ? 0 : Mout;   // with pruning the Horner kernel sets it
        } else if (d == 1) {
          q = kQLinear;
          nt = Mout;
        } else if (D <= row_dmax) {
          q = D;
          nt = Mout;
        } else if (D <= T.dmax) {
          q = kQPairs;
          nt = Mout;
        } else {
          atomicOr(status, kStatusUnsupported);
        }
      }
    }
    A.post_nterms[item] = nt;
  }
  int rank_in_warp = 0;
  for (int qq = 0; qq < kComposeQueues; ++qq) {
    const unsigned m = __ballot_sync(0xffffffffu, q == qq);
    if (q == qq) rank_in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) s_wcnt[warp][qq] = __popc(m);
  }
  __syncthreads();
  if (threadIdx.x < kComposeQueues) {
    const int qq = threadIdx.x;
    int run = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {   // exclusive scan over warps
      const int c = s_wcnt[w][qq];
      s_wcnt[w][qq] = run;
      run += c;
    }
    s_base[qq] = run ? atomicAdd(&S.qcount[qq], run) : 0;
  }
  __syncthreads();
  if (q >= 0) S.queue[(int64_t)q * S.qcap + s_base[q] + s_wcnt[warp][q] + rank_in_warp] = (int)item;
}

// ------------------------------------------------------------ row convolution
constexpr int kRowWarps = 4;    // warps sharing one 32-item group
constexpr int kRowBlocks = 8;   // resident blocks per SM (registers and shared memory)

// Load one bound of the 32 items of a lane group into row layout:
// s = (pre - lo*[K=0]) / (hi - lo) in round-to-nearest; returns this warp's
// share of sum|s| (rounded up).  Warp `half` (of kRowWarps) takes every
// kRowWarps-th group
// of 8 input monomials.
__device__ float load_rows(const ComposeArgs& A, const RowTable& R, const float* P, int Mpre,
                           float Lo, float inv, int half, float* s) {
  const int h = A.h;
  float l1 = 0.0f;
  for (int r0 = 8 * half; r0 < R.m_in; r0 += 8 * kRowWarps) {
    float v[8];
    int pos[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + i;
      v[i] = r < Mpre ? __ldg(P + (int64_t)r * h) : 0.0f;
      pos[i] = r < R.m_in ? __ldg(R.pos_in + r) : -1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (pos[i] < 0) continue;
      float x = v[i];
      if (r0 + i == 0) x = __fsub_rn(x, Lo);
      x = __fmul_rn(x, inv);
      s[pos[i]] = x;
      l1 = __fadd_ru(l1, fabsf(x));
    }
  }
  return l1;
}

// Output rows [row_b, row_e) of one bound (UP: upper polynomial) of the
// items of a warp: per row, the row-pair convolutions, then the coefficients
// a1*s + a2*s^2 of the row's monomials (the constant term only in c0).
template <bool UP>
__device__ void rows_range(const Tables& T, const ComposeArgs& A, const RowTable& R, int D,
                           int row_b, int row_e, int row_step, bool valid, float a1, float a2,
                           const float* s, float* Q, float* c0_out, float* rem_out) {
  const int h = A.h;
  const int Mout = T.mcount[min(2 * D, A.cap)];
  const bool no_trunc = 2 * D <= A.cap;   // every output monomial is kept
  float rem = 0.0f;
  for (int row = row_b; row < row_e; row += row_step) {
    const int4 hd = __ldg(R.hdr + row);
    const int Lout = hd.w & 0xff, in_len = (hd.w >> 8) & 0xff;
    const int in_off = __ldg(R.in_off + row);
    float acc[2 * kRowLen - 1];
#pragma unroll
    for (int c = 0; c < 2 * kRowLen - 1; ++c) acc[c] = 0.0f;
    const int has_diag = (hd.w >> 16) & 1;
    const int off_end = hd.y - has_diag;
    if (hd.x < off_end) {
      int4 pr = __ldg(R.pairs + hd.x);
      for (int k = hd.x; k < off_end; ++k) {
        const int4 nx = k + 1 < off_end ? __ldg(R.pairs + k + 1) : pr;   // prefetch
        switch (pr.w) {
          BERN_CONV_ALL_CASES
          default: break;
        }
        pr = nx;
      }
    }
    if (has_diag) {
      const int4 pr = __ldg(R.pairs + off_end);
      switch (pr.z & 15) {
        BERN_DIAG_CASES
        default: break;
      }
    }
    const int* __restrict__ rk = R.out_ranks + hd.z;   // the row's output ranks
#pragma unroll
    for (int c = 0; c < 2 * kRowLen - 1; ++c) {
      if (c >= Lout) break;
      const float sq = acc[c];            // (s^2)_K, directed
      const float lin = c < in_len ? s[in_off + c] : 0.0f;
      const float v = dfma<UP>(a2, sq, UP ? __fmul_ru(a1, lin) : __fmul_rd(a1, lin));
      if (row == 0 && c == 0) {
        *c0_out = v;                      // the constant term is finished by the caller
      } else if (no_trunc || __ldg(rk + c) < Mout) {
        if (valid) Q[(int64_t)__ldg(rk + c) * h] = v;
      } else {
        rem = UP ? __fadd_ru(rem, fmaxf(v, 0.0f)) : __fadd_rd(rem, fminf(v, 0.0f));
      }
    }
  }
  *rem_out = rem;
}

// A block of kRowWarps warps squares one bound (UP: upper) of 32 queued items
// (one lane per item); the warps share the items' inputs in shared memory and
// take the output rows in turn.
template <bool UP>
__global__ void __launch_bounds__(32 * kRowWarps, kRowBlocks)
k_compose_rows(Tables T, ComposeArgs A, ComposeScratch S, int row_dmax, int sstride,
               int* status) {
  extern __shared__ float smem[];
  __shared__ float s_l1[kRowWarps][32], s_rem[kRowWarps][32], s_c0[32];
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;
  float* s = smem + (size_t)lane * sstride;
  for (int task = blockIdx.x;; task += gridDim.x) {
    int D = -1, chunk = task;
    for (int d = 0; d <= row_dmax; ++d) {
      const int nc = (S.qcount[d] + 31) >> 5;
      if (chunk < nc) {
        D = d;
        break;
      }
      chunk -= nc;
    }
    if (D < 0) break;
    const int idx = chunk * 32 + lane;
    const bool valid = idx < S.qcount[D];
    const int64_t item = valid ? S.queue[(int64_t)D * S.qcap + idx] : 0;
    const RowTable R = T.row[D];
    const float Lo = valid ? A.lo[item] : -1.0f;
    const float Hi = valid ? A.hi[item] : 1.0f;
    const float inv = 1.0f / (Hi - Lo);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    if (valid) {
      const float* cf = A.coef + item * kCoefStride;
      a0 = cf[0];
      a1 = cf[1];
      a2 = cf[2];
      if (a2 < 0.0f) atomicOr(status, kStatusUnsupported);   // excluded by convexity
    }
    const int Mpre = valid ? A.pre_nterms[item] : 0;
    const float* P = (UP ? A.pre_up : A.pre_lo) + A.base(valid ? item : 0, A.pre_ld);
    s_l1[half][lane] = load_rows(A, R, P, Mpre, Lo, inv, half, s);
    __syncthreads();
    float* Q = (UP ? A.post_up : A.post_lo) + A.base(valid ? item : 0, A.post_ld);
    float c0 = 0.0f, rem = 0.0f;
    rows_range<UP>(T, A, R, D, half, R.n_out_rows, kRowWarps, valid, a1, a2, s, Q, &c0, &rem);
    s_rem[half][lane] = rem;
    if (!half) s_c0[lane] = c0;
    __syncthreads();
    if (!half && valid) {
      // constant term: a0 + (the row-0 value without a0) + Lip*eta + remainder
      float l1 = s_l1[0][lane], remt = s_rem[0][lane];
#pragma unroll
      for (int w = 1; w < kRowWarps; ++w) {
        l1 = __fadd_ru(l1, s_l1[w][lane]);
        remt = UP ? __fadd_ru(remt, s_rem[w][lane]) : __fadd_rd(remt, s_rem[w][lane]);
      }
      const float eta = __fmul_ru(5.0f * kU, l1);
      const float lip = __fmaf_ru(2.0f * a2, __fadd_ru(1.0f, eta), fabsf(a1));
      float v;
      if (UP) {
        v = __fadd_ru(__fadd_ru(__fadd_ru(s_c0[lane], a0), __fmul_ru(lip, eta)), remt);
      } else {
        v = __fsub_rd(__fadd_rd(s_c0[lane], a0), __fmul_ru(lip, eta));
        v = __fadd_rd(__fsub_rd(v, A.eps[item]), remt);
      }
      Q[0] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
    __syncthreads();   // the next task reuses the shared inputs
  }
}

// ------------------------------------------------------------ elementwise items
// Identity items copy pre to post: a lane per queue entry (32 consecutive
// entries per warp, so neighbouring lanes touch neighbouring neurons), the
// warps of a block over the coefficient rows.
__global__ void __launch_bounds__(256)
k_compose_copy(ComposeArgs A, ComposeScratch S) {
  const int cnt = S.qcount[kQIdent];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t h = A.h;
  for (int64_t t0 = (int64_t)blockIdx.x * 32; t0 < cnt; t0 += (int64_t)gridDim.x * 32) {
    const int64_t t = t0 + lane;
    if (t >= cnt) continue;
    const int64_t item = S.queue[(int64_t)kQIdent * S.qcap + t];
    const int nt = A.pre_nterms[item];
    const float* su = A.pre_up + A.base(item, A.pre_ld);
    const float* sl = A.pre_lo + A.base(item, A.pre_ld);
    float* du = A.post_up + A.base(item, A.post_ld);
    float* dl = A.post_lo + A.base(item, A.post_ld);
    // four rows of each bound in flight per round
    int r = warp;
    for (; r + 3 * nw < nt; r += 4 * nw) {
      float vu[4], vl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        vu[q] = su[(r + q * nw) * h];
        vl[q] = sl[(r + q * nw) * h];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        du[(r + q * nw) * h] = vu[q];
        dl[(r + q * nw) * h] = vl[q];
      }
    }
    for (; r < nt; r += nw) {
      du[r * h] = su[r * h];
      dl[r * h] = sl[r * h];
    }
  }
}

// Order-1 items: a0 + a1*s~ for both bounds, one warp per item.
__global__ void __launch_bounds__(256)
k_compose_linear(ComposeArgs A, ComposeScratch S, int* status) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int n_lin = S.qcount[kQLinear];
  const int h = A.h;
  for (int t = gw; t < n_lin; t += nw) {
    const int64_t item = S.queue[(int64_t)kQLinear * S.qcap + t];
    const int Mpre = A.pre_nterms[item];
    const float* Pu = A.pre_up + A.base(item, A.pre_ld);
    const float* Pl = A.pre_lo + A.base(item, A.pre_ld);
    float* Qu = A.post_up + A.base(item, A.post_ld);
    float* Ql = A.post_lo + A.base(item, A.post_ld);
    const float Lo = A.lo[item], Hi = A.hi[item];
    const float inv = 1.0f / (Hi - Lo);
    const float* cf = A.coef + item * kCoefStride;
    const float a0 = cf[0], a1 = cf[1];
    const int Mout = A.post_nterms[item];     // the graded prefix of Mpre's degree
    float lu = 0.0f, ll = 0.0f, cu0 = 0.0f, cl0 = 0.0f;
    for (int r = lane; r < Mout; r += 32) {
      float vu = r < Mpre ? Pu[(int64_t)r * h] : 0.0f, vl = r < Mpre ? Pl[(int64_t)r * h] : 0.0f;
      if (r == 0) {
        vu = __fsub_rn(vu, Lo);
        vl = __fsub_rn(vl, Lo);
      }
      vu = __fmul_rn(vu, inv);
      vl = __fmul_rn(vl, inv);
      lu = __fadd_ru(lu, fabsf(vu));
      ll = __fadd_ru(ll, fabsf(vl));
      const float cu = __fmaf_ru(a1, vu, r == 0 ? a0 : 0.0f);
      const float cl = __fmaf_rd(a1, vl, r == 0 ? a0 : 0.0f);
      if (r == 0) {
        cu0 = cu;
        cl0 = cl;
      } else {
        Qu[(int64_t)r * h] = cu;
        Ql[(int64_t)r * h] = cl;
      }
    }
    lu = warp_dsum<true>(lu);
    ll = warp_dsum<true>(ll);
    if (lane == 0) {
      const float lip = fabsf(a1);
      const float eu = __fmul_ru(5.0f * kU, lu), el = __fmul_ru(5.0f * kU, ll);
      const float vu = __fadd_ru(cu0, __fmul_ru(lip, eu));
      const float vl = __fsub_rd(__fsub_rd(cl0, __fmul_ru(lip, el)), A.eps[item]);
      Qu[0] = vu;
      Ql[0] = vl;
      if (!isfinite(vu) || !isfinite(vl)) atomicOr(status, kStatusNonFinite);
    }
  }
}

// ------------------------------------------------------------ pair-list squaring
// Order-2 items outside the row path: one block per item, threads over output
// monomials, symmetric pair lists (I <= J, I + J = K) from the host tables.
__global__ void __launch_bounds__(256)
k_compose_pairs(Tables T, ComposeArgs A, ComposeScratch S, int* status) {
  extern __shared__ float smem[];
  __shared__ float red[32];
  __shared__ float c0[2];
  const int count = S.qcount[kQPairs];
  for (int t = blockIdx.x; t < count; t += gridDim.x) {
    const int64_t item = S.queue[(int64_t)kQPairs * S.qcap + t];
    const int Mpre = A.pre_nterms[item];
    const int Dpre = degree_of(T, Mpre);
    const int Mp = T.mcount[Dpre];
    const int Dfull = 2 * Dpre;
    const int Mout = T.mcount[min(Dfull, A.cap)];
    const int Mfull = T.mcount[Dfull];
    const int h = A.h;
    const float* Pu = A.pre_up + A.base(item, A.pre_ld);
    const float* Pl = A.pre_lo + A.base(item, A.pre_ld);
    float* Qu = A.post_up + A.base(item, A.post_ld);
    float* Ql = A.post_lo + A.base(item, A.post_ld);
    const float L = A.lo[item], H = A.hi[item];
    const float inv = 1.0f / (H - L);
    float* su = smem;
    float* sl = smem + A.pre_cap;
    float au = 0.0f, al = 0.0f;
    for (int r = threadIdx.x; r < Mp; r += blockDim.x) {
      float vu = r < Mpre ? Pu[(int64_t)r * h] : 0.0f, vl = r < Mpre ? Pl[(int64_t)r * h] : 0.0f;
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
    const float* cf = A.coef + item * kCoefStride;
    const float a0 = cf[0], a1 = cf[1], a2 = cf[2];
    const bool a2pos = a2 >= 0.0f;
    const PairTable pt = T.sq[Dpre];
    float remU = 0.0f, remL = 0.0f;
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
      const float sqU = __fadd_ru(diagU, 2.0f * offU);
      const float sqL = __fadd_rd(diagL, 2.0f * offL);
      const float cu = __fmaf_ru(a2, a2pos ? sqU : sqL,
                                 __fmaf_ru(a1, K < Mp ? su[K] : 0.0f, K == 0 ? a0 : 0.0f));
      const float cl = __fmaf_rd(a2, a2pos ? sqL : sqU,
                                 __fmaf_rd(a1, K < Mp ? sl[K] : 0.0f, K == 0 ? a0 : 0.0f));
      if (K == 0) {
        c0[0] = cu;
        c0[1] = cl;
      } else if (K < Mout) {
        Qu[(int64_t)K * h] = cu;
        Ql[(int64_t)K * h] = cl;
      } else {
        remU = __fadd_ru(remU, fmaxf(cu, 0.0f));
        remL = __fadd_rd(remL, fminf(cl, 0.0f));
      }
    }
    __syncthreads();
    remU = block_dsum<true>(remU, red);
    __syncthreads();
    remL = block_dsum<false>(remL, red);
    if (threadIdx.x == 0) {
      const float lipu = __fmaf_ru(2.0f * fabsf(a2), __fadd_ru(1.0f, eta_u), fabsf(a1));
      const float lipl = __fmaf_ru(2.0f * fabsf(a2), __fadd_ru(1.0f, eta_l), fabsf(a1));
      float cu = __fadd_ru(__fadd_ru(c0[0], __fmul_ru(lipu, eta_u)), remU);
      float cl = __fsub_rd(c0[1], __fmul_ru(lipl, eta_l));
      cl = __fadd_rd(__fsub_rd(cl, A.eps[item]), remL);
      Qu[0] = cu;
      Ql[0] = cl;
      if (!isfinite(cu) || !isfinite(cl)) atomicOr(status, kStatusNonFinite);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ launcher
cudaError_t launch_compose(const Launch& L, const Tables& T, const ComposeScratch& S,
                           int64_t n_boxes, int h, int cap, float tau, const int8_t* kind,
                           const float* coef, const float* eps, const uint8_t* degrees,
                           int global_d, const float* lo, const float* hi, const float* pre_up,
                           const float* pre_lo, int64_t pre_ld, const int32_t* pre_nterms,
                           float* post_up, float* post_lo, int64_t post_ld,
                           int32_t* post_nterms, int64_t pre_cap) {
  const int64_t n_items = n_boxes * h;
  if (n_items == 0) return cudaSuccess;
  if (pre_cap <= 0) pre_cap = pre_ld;
  if (!(tau >= 0.0f) || n_items > S.qcap || n_items > INT32_MAX || pre_cap > pre_ld)
    return cudaErrorInvalidValue;
  const bool in_place = post_up == pre_up && post_lo == pre_lo;
  if (in_place && post_ld != pre_ld) return cudaErrorInvalidValue;
  ComposeArgs A{cap, tau, h, kind, coef, eps, degrees, global_d, lo, hi, pre_up, pre_lo, pre_ld,
                pre_nterms, post_up, post_lo, post_ld, post_nterms, pre_cap};
  // the largest input degree any item of this call can have
  int Dmax = 0;
  while (Dmax < kMaxTableDegree && num_monomials(T.n, Dmax + 1) >= 0 &&
         num_monomials(T.n, Dmax + 1) <= pre_cap)
    ++Dmax;
  const int row_dmax = std::min(std::min(T.row_dmax, row_path_max_degree(T.n)), Dmax);
  cudaError_t e = cudaMemsetAsync(S.qcount, 0, kComposeQueues * sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  k_compose_queue<<<(unsigned)((n_items + 1023) / 1024), 1024, 0, L.stream>>>(
      T, A, n_items, row_dmax, S, L.status);
  ++*L.launches;
  // order-2 items exist only with order 2 somewhere in the plan (with pruning
  // they go to the Horner kernel)
  const bool order2 = tau == 0.0f && (degrees != nullptr || global_d == 2);
  // row-convolution kernels (one per bound): persistent blocks of 2 warps
  // per 32 items; the per-lane stride is odd so that lanes reading the same
  // offset hit distinct banks
  const int sstride = (int)num_monomials(T.n, row_dmax) | 1;
  const size_t smem = (size_t)32 * sstride * sizeof(float);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_compose_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_compose_rows<false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t tasks = n_items / 32 + row_dmax + 1;
  const int blocks = (int)std::min<int64_t>(tasks, device_sms(L) * kRowBlocks);
  if (order2) {
    k_compose_rows<true><<<blocks, 32 * kRowWarps, smem, L.stream>>>(T, A, S, row_dmax, sstride,
                                                                     L.status);
    k_compose_rows<false><<<blocks, 32 * kRowWarps, smem, L.stream>>>(T, A, S, row_dmax,
                                                                      sstride, L.status);
    *L.launches += 2;
  }
  if (!in_place) {   // in place, an identity item's outputs are its inputs
    k_compose_copy<<<(unsigned)std::min<int64_t>((n_items + 31) / 32, device_sms(L) * 16), 256, 0,
                     L.stream>>>(A, S);
    ++*L.launches;
  }
  // order-1 items exist only with order 1 somewhere in the plan (with pruning
  // they go to the Horner kernel)
  if (tau == 0.0f && (degrees != nullptr || global_d == 1)) {
    k_compose_linear<<<(unsigned)std::min<int64_t>((n_items + 7) / 8, device_sms(L) * 16), 256,
                       0, L.stream>>>(A, S, L.status);
    ++*L.launches;
  }
  // pair-list kernel for order-2 items beyond the row path
  if (order2 && Dmax > row_dmax) {
    const size_t psmem = 2 * (size_t)pre_cap * sizeof(float);
    if (psmem > 200 * 1024) return cudaErrorInvalidValue;
    if (psmem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_compose_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem);
      if (e != cudaSuccess) return e;
    }
    k_compose_pairs<<<(unsigned)std::min<int64_t>(n_items, device_sms(L) * 8), 256, psmem, L.stream>>>(
        T, A, S, L.status);
    ++*L.launches;
  }
  // Horner kernels for orders >= 3, and for every order when pruning
  if (tau > 0.0f || global_d >= 3) {
    e = launch_compose_horner(L, T, S, A, Dmax);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace bern
