// One hidden layer in one launch: from the layer's pre-activation bounds to
// the NEXT layer's pre-activation bounds, with everything in between kept in
// shared memory.  Per box (one block per box, persistent blocks taking boxes
// from a counter):
//
//   a2  stability screen and Bernstein enclosure (Sec. 5.1 Step 1, Def. 2)
//   a3  ReLU case and order-d Bernstein coefficients (Step 2, Props. 1-2)
//   a4  composition B(s(t)) for orders 1 and 2 (Step 3, eqs. post_bounds_1/2)
//   a1  the next layer's step (Sec. 5.2, eqs. upper/lower_bounds_layer)
//
// so a post-activation polynomial never goes to HBM: the block reads the
// layer block pre[M x h] of its box once and writes next[M' x h'] once, whole
// 32-byte sectors at a time.  The arithmetic is that of the per-step kernels
// (k_stable_screen, k_enclose, k_compose_rows / k_compose_linear,
// k_affine_wide): every value is rounded in the same direction, in the same
// order, except the cap-truncation remainder (summed per warp here) and the
// next layer's affine step, whose sum runs over the live neurons in index
// order (dead neurons add exact zeros).
//
// Shared memory per block:
//   S     both bounds of every neuron's polynomial in row layout (the
//         monomials sharing the exponents of t_1..t_{n-1} contiguous), raw
//         pre-activation coefficients, then s = (pre - lo)/(hi - lo) for the
//         unstable neurons; stride ss (odd) per (bound, neuron)
//   W     the next layer's weights transposed, [h][hnp]
//   union the enclosure grids (one per warp), then the output tiles
//   per-neuron scalars and lists
//
// Composition (order 2) maps lanes to (neuron, bound) slots of the unstable
// neurons of the box, upper and lower bounds of the same warp sharing one
// instruction stream: a lower-bound lane negates one operand and rounds up,
// which yields exactly the negated round-down value (RU(-x) = -RD(x)).  The
// output is produced by tiles of whole output rows; each tile's (upper,
// lower) values of all live neurons are turned into (midpoint, radius)
// pairs and multiplied by the next layer's weights at once.
#include <algorithm>

#include "compose_common.cuh"
#include "enclose_impl.cuh"
#include "row_conv.cuh"

namespace bern {

namespace {

constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / 32;

struct LayerArgs {
  int n, h, d, cap, hn;
  int64_t n_boxes;
  const float* pre_up;
  const float* pre_lo;
  int64_t pre_ld;
  const int32_t* pre_nt;
  const float* Wn;       // next layer [hn x h] row-major
  const float* bn;       // [hn]
  float* nx_up;
  float* nx_lo;
  int64_t nx_ld;
  int32_t* nx_nt;
  int* counter;          // boxes taken so far (zeroed before the launch)
  // shared-memory layout, in 4-byte words
  int ss, hnp, offW, offU, uni, offN, rem_on;
  int mcap;              // M(n, D_pre): the most monomials a box may have (<= ss)
};

// Block-wide stable compaction of the indices whose flag is set (every
// thread calls it; thread t carries index t).  Returns the count.
__device__ __forceinline__ int block_compact(bool flag, int* list, int* s_wcount) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) s_wcount[warp] = __popc(bal);
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kLWarps; ++w) {
    const int c = s_wcount[w];
    if (w < warp) base += c;
    total += c;
  }
  if (flag) list[base + __popc(bal & ((1u << lane) - 1u))] = threadIdx.x;
  __syncthreads();
  return total;
}

// The affine step of the next layer on one tile: outputs (entry e, neuron m')
// for the E tile entries (ranks rank_of(e)), inputs the nv live neurons'
// (midpoint, radius) pairs in tile columns.  TM = 4: register tiles of
// 4 entries x 4 next-layer neurons (float4 weight loads); TM = 1: one
// neuron per thread tile.
template <int TM, class RankOf>
__device__ __forceinline__ void tile_affine(const LayerArgs& A, int64_t b, const float* sW,
                                            const int* lV, int nv, const float* tC,
                                            const float* tR, int vs, int E, int e_b,
                                            RankOf rank_of, int Mkeep) {
  const int ntile_e = (E + 3) >> 2;
  const int ntile_m = TM == 4 ? (A.hnp >> 2) : A.hn;
  for (int tt = threadIdx.x; tt < ntile_e * ntile_m; tt += kLThreads) {
    const int eg = tt / ntile_m, mg = tt - eg * ntile_m;
    float uc[4][TM], lc[4][TM], rad[4][TM];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        uc[k][i] = 0.0f;
        lc[k][i] = 0.0f;
        rad[k][i] = 0.0f;
      }
    const float* pc = tC + (4 * eg) * vs;
    const float* pr = tR + (4 * eg) * vs;
    for (int vi = 0; vi < nv; ++vi) {
      const int j = lV[vi];
      float w[TM];
      if constexpr (TM == 4) {
        const float4 w4 = *reinterpret_cast<const float4*>(sW + j * A.hnp + 4 * mg);
        w[0] = w4.x;
        w[1] = w4.y;
        w[2] = w4.z;
        w[3] = w4.w;
      } else {
        w[0] = sW[j * A.hnp + mg];
      }
      float c[4], r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[k] = pc[k * vs + vi];
        r[k] = pr[k * vs + vi];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          uc[k][i] = __fmaf_ru(w[i], c[k], uc[k][i]);
          lc[k][i] = __fmaf_rd(w[i], c[k], lc[k][i]);
          rad[k][i] = __fmaf_ru(fabsf(w[i]), r[k], rad[k][i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int el = 4 * eg + k;
      if (el >= E) continue;
      const int e = e_b + el;
      const int rank = rank_of(e);
      if (rank == 0 || rank >= Mkeep) continue;   // rank 0 is finished last
      const int64_t o = (b * A.nx_ld + rank) * A.hn;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int mp = TM == 4 ? 4 * mg + i : mg;
        if (mp < A.hn) {
          A.nx_up[o + mp] = __fadd_ru(uc[k][i], rad[k][i]);
          A.nx_lo[o + mp] = __fsub_rd(lc[k][i], rad[k][i]);
        }
      }
    }
  }
}

// (upper, lower) tile values -> (midpoint, radius), as the affine kernels
// form them from their inputs.
__device__ __forceinline__ void tile_to_midrad(float* tU, float* tL, int E, int nv, int vs) {
  for (int idx = threadIdx.x; idx < E * nv; idx += kLThreads) {
    const int el = idx / nv, vi = idx - el * nv;
    const float u = tU[el * vs + vi], l = tL[el * vs + vi];
    const float c = __fmaf_rn(0.5f, u, 0.5f * l);
    tU[el * vs + vi] = c;
    tL[el * vs + vi] = fmaxf(__fsub_ru(u, c), __fsub_ru(c, l));
  }
}

// Up to order 4 the layer blocks are small enough for four blocks per SM (64
// registers); above, the block of a box takes half an SM's shared memory.
template <int LB>
__global__ void __launch_bounds__(kLThreads, LB <= 4 ? 4 : 2)
k_layer(Tables T, LayerArgs A, const float2* __restrict__ rs, int* status) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int sh_box, sh_M, sh_Mnext, sh_tile_end, sh_row_end;
  __shared__ int s_wcount[kLWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = A.h, hn = A.hn, ss = A.ss;
  float* sS = smem;
  float* sW = smem + A.offW;
  float* sUn = smem + A.offU;
  float* n_lo = smem + A.offN;
  float* n_hi = n_lo + h;
  float* n_a0 = n_hi + h;
  float* n_a1 = n_a0 + h;
  float* n_a2 = n_a1 + h;
  float* n_eps = n_a2 + h;
  int* n_kind = reinterpret_cast<int*>(n_eps + h);
  int* n_nt = n_kind + h;
  int* lU = n_nt + h;
  int* lV = lU + h;
  int* lC = lV + h;
  int* n_col = lC + h;
  float* s_eta = reinterpret_cast<float*>(n_col + h);    // [2h] per slot
  float* s_c0 = s_eta + 2 * h;                            // [2h] per slot
  float* s_rem = s_c0 + 2 * h;                            // [kLWarps][2h] if rem_on
  const int n = A.n;

  // the next layer's weights, transposed (input-neuron major)
  for (int idx = tid; idx < h * A.hnp; idx += kLThreads) {
    const int j = idx / A.hnp, mp = idx - j * A.hnp;
    sW[idx] = mp < hn ? A.Wn[(int64_t)mp * h + j] : 0.0f;
  }
  for (;;) {
    __syncthreads();                       // the previous box is finished
    if (tid == 0) {
      sh_box = atomicAdd(A.counter, 1);
      sh_M = 0;
      sh_Mnext = 1;
    }
    __syncthreads();
    const int64_t b = sh_box;
    if (b >= A.n_boxes) break;

    // ---- term counts of the box's pre-activation polynomials
    for (int m = tid; m < h; m += kLThreads) {
      int v = A.pre_nt[b * h + m];
      if (v < 0 || v > A.pre_ld) {
        atomicOr(status, kStatusInvalid);
        v = 0;
      }
      n_nt[m] = v;
      atomicMax(&sh_M, v);
    }
    __syncthreads();
    const int Mb = sh_M;
    const int Db = Mb <= T.mexps ? (int)T.deg_of[Mb] : kMaxTableDegree;
    if (Db > T.row_dmax) {                 // excluded by the launcher
      if (tid == 0) atomicOr(status, kStatusUnsupported);
      continue;
    }
    const RowTable R = T.row[Db];
    const int m_in = R.m_in;               // M(n, Db) >= Mb
    if (m_in > A.mcap) {                   // a term count past the layer's degree
      if (tid == 0) atomicOr(status, kStatusInvalid);
      continue;
    }

    // ---- the layer block into row layout (entries past a term count are 0)
    {
      const float* gu = A.pre_up + (b * A.pre_ld) * h;
      const float* gl = A.pre_lo + (b * A.pre_ld) * h;
      constexpr int kB = 4;
      for (int i0 = tid; i0 < m_in * h; i0 += kLThreads * kB) {
        float u[kB], l[kB];
        int at[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) {
          const int idx = i0 + q * kLThreads;
          u[q] = 0.0f;
          l[q] = 0.0f;
          at[q] = -1;
          if (idx < m_in * h) {
            const int r = idx / h, m = idx - r * h;
            if (r < n_nt[m]) {
              u[q] = __ldg(gu + idx);
              l[q] = __ldg(gl + idx);
            }
            at[q] = m * ss + __ldg(R.pos_in + r);
          }
        }
#pragma unroll
        for (int q = 0; q < kB; ++q)
          if (at[q] >= 0) {
            sS[at[q]] = u[q];
            sS[h * ss + at[q]] = l[q];
          }
      }
    }
    __syncthreads();

    // ---- stability screen (coefficient signs; every monomial is in [0,1])
    bool cand = false;
    if (tid < h) {
      const int m = tid, nt = n_nt[m];
      const float* pu = sS + m * ss;
      const float* pl = sS + (h + m) * ss;
      float l = 0.0f, u = 0.0f;
      if (nt > 0) {
        l = pl[0];
        u = pu[0];
        for (int r = 1; r < nt; ++r) {
          const int p = __ldg(R.pos_in + r);
          l = __fadd_rd(l, fminf(pl[p], 0.0f));
          u = __fadd_ru(u, fmaxf(pu[p], 0.0f));
        }
      }
      if (!(isfinite(l) && isfinite(u)) || (u > 0.0f && l < 0.0f)) {
        cand = true;
      } else {
        n_kind[m] = u <= 0.0f ? 0 : 1;
        n_lo[m] = l;
        n_hi[m] = u;
      }
    }
    const int nc = block_compact(cand, lC, s_wcount);

    // ---- Bernstein enclosure of the undecided neurons: a warp per polynomial
    {
      const int G = ipow(LB + 1, n);
      float* grid = sUn + (size_t)warp * G;
      for (int p = warp; p < 2 * nc; p += kLWarps) {
        const int m = lC[p >> 1];
        const bool up = p & 1;
        const int nt = n_nt[m];
        const float v =
            up ? enclose_warp<LB, true, true>(sS + m * ss, 1, nt, n, T, rs, grid, R.pos_in)
               : enclose_warp<LB, false, true>(sS + (h + m) * ss, 1, nt, n, T, rs, grid,
                                                R.pos_in);
        if (lane == 0) {
          (up ? n_hi : n_lo)[m] = v;
          if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- ReLU cases and coefficients (a thread per undecided neuron)
    for (int t = tid; t < nc; t += kLThreads) {
      const int m = lC[t];
      float a[kCoefStride];
      float e = 0.0f;
      a[0] = a[1] = a[2] = 0.0f;
      const int k = relu_item(n_lo[m], n_hi[m], A.d, a, &e, status);
      n_kind[m] = k;
      if (k == 2) {
        n_a0[m] = a[0];
        n_a1[m] = a[1];
        n_a2[m] = A.d >= 2 ? a[2] : 0.0f;
        n_eps[m] = e;
        if (A.d >= 2 && a[2] < 0.0f) atomicOr(status, kStatusUnsupported);   // convexity
      }
    }
    __syncthreads();

    // ---- unstable and live neuron lists, next term count
    const int kind_t = tid < h ? n_kind[tid] : 0;
    const int nu = block_compact(kind_t == 2, lU, s_wcount);
    const int nv = block_compact(kind_t >= 1, lV, s_wcount);
    const int Dout2 = min(2 * Db, A.cap);
    const int Mout = A.d >= 2 ? T.mcount[Dout2] : T.mcount[min(Db, A.cap)];
    if (tid < h) {
      int pnt = 0;
      if (kind_t == 1) pnt = n_nt[tid];
      if (kind_t == 2) {
        // order 1 keeps each neuron's own degree (its graded prefix)
        pnt = A.d >= 2 ? Mout : T.mcount[min((int)T.deg_of[n_nt[tid]], A.cap)];
      }
      if (pnt > 1) atomicMax(&sh_Mnext, pnt);
    }
    for (int vi = tid; vi < nv; vi += kLThreads) n_col[lV[vi]] = vi;
    __syncthreads();
    const int Mnext = sh_Mnext;
    if (Mnext > A.nx_ld) {
      if (tid == 0) atomicOr(status, kStatusCapacity);
      continue;
    }
    for (int mp = tid; mp < hn; mp += kLThreads) A.nx_nt[b * hn + mp] = Mnext;

    // ---- s = (pre - lo*[K=0]) / (hi - lo) in place for the unstable slots,
    // and eta = 5u * sum|s| (summed as the per-step kernels sum it)
    if (A.d >= 2) {
      float* part = sUn;                    // [2h][4] partial sums
      for (int t = tid; t < 8 * nu; t += kLThreads) {
        const int slot = t >> 2, half = t & 3;
        const int bound = slot >= nu;
        const int m = lU[slot - bound * nu];
        const float Lo = n_lo[m], Hi = n_hi[m];
        const float inv = 1.0f / (Hi - Lo);
        float* P = sS + (bound * h + m) * ss;
        float l1 = 0.0f;
        for (int r0 = 8 * half; r0 < m_in; r0 += 32) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = r0 + i;
            if (r >= m_in) break;
            const int p = __ldg(R.pos_in + r);
            float x = P[p];
            if (r == 0) x = __fsub_rn(x, Lo);
            x = __fmul_rn(x, inv);
            P[p] = x;
            l1 = __fadd_ru(l1, fabsf(x));
          }
        }
        part[slot * 4 + half] = l1;
      }
      __syncthreads();
      for (int slot = tid; slot < 2 * nu; slot += kLThreads) {
        float l1 = part[slot * 4];
#pragma unroll
        for (int w = 1; w < 4; ++w) l1 = __fadd_ru(l1, part[slot * 4 + w]);
        s_eta[slot] = __fmul_ru(5.0f * kU, l1);
      }
    } else {
      // order 1: a warp per slot, lanes over the graded ranks of the
      // neuron's own prefix, a warp sum
      for (int slot = warp; slot < 2 * nu; slot += kLWarps) {
        const int bound = slot >= nu;
        const int m = lU[slot - bound * nu];
        const float Lo = n_lo[m], Hi = n_hi[m];
        const float inv = 1.0f / (Hi - Lo);
        float* P = sS + (bound * h + m) * ss;
        const int Mo = T.mcount[min((int)T.deg_of[n_nt[m]], A.cap)];
        float l1 = 0.0f;
        for (int r = lane; r < Mo; r += 32) {
          const int p = __ldg(R.pos_in + r);
          float x = P[p];
          if (r == 0) x = __fsub_rn(x, Lo);
          x = __fmul_rn(x, inv);
          P[p] = x;
          l1 = __fadd_ru(l1, fabsf(x));
        }
        l1 = warp_dsum<true>(l1);
        if (lane == 0) s_eta[slot] = __fmul_ru(5.0f * kU, l1);
      }
    }
    if (A.rem_on)
      for (int i = tid; i < kLWarps * 2 * h; i += kLThreads) s_rem[i] = 0.0f;
    __syncthreads();

    // ---- composition and the next layer's affine step, tile by tile
    const int vs = nv | 1;
    const int Rcap = (A.uni / (2 * vs)) & ~3;
    float* tU = sUn;
    float* tL = sUn + Rcap * vs;
    if (A.d >= 2 && nu > 0) {
      // output tiles of whole rows of the row table
      const int nrows = R.n_out_rows;
      const int m_full = T.mcount[2 * Db];
      int row_b = 0;
      while (row_b < nrows) {
        if (tid == 0) {
          const int e_b0 = __ldg(&R.hdr[row_b].z);
          int re = row_b + 1;
          while (re < nrows && __ldg(&R.hdr[re].z) + (__ldg(&R.hdr[re].w) & 0xff) - e_b0 <= Rcap)
            ++re;
          sh_row_end = re;
          sh_tile_end = re < nrows ? __ldg(&R.hdr[re].z) : m_full;
        }
        __syncthreads();
        const int row_e = sh_row_end;
        const int e_b = __ldg(&R.hdr[row_b].z);
        const int E = sh_tile_end - e_b;
        // identity neurons: their own coefficients (ranks below m_in), else 0
        for (int idx = tid; idx < E * nv; idx += kLThreads) {
          const int el = idx / nv, vi = idx - el * nv;
          const int m = lV[vi];
          if (n_kind[m] != 1) continue;
          const int rank = __ldg(R.out_ranks + e_b + el);
          float u = 0.0f, l = 0.0f;
          if (rank < m_in) {
            const int p = __ldg(R.pos_in + rank);
            u = sS[m * ss + p];
            l = sS[(h + m) * ss + p];
          }
          tU[el * vs + vi] = u;
          tL[el * vs + vi] = l;
        }
        // unstable neurons: a warp per (group of 32 slots, output row)
        const int ngroups = (2 * nu + 31) >> 5;
        const int nrt = row_e - row_b;
        for (int unit = warp; unit < ngroups * nrt; unit += kLWarps) {
          const int g = unit / nrt, row = row_b + (unit - g * nrt);
          const int slot = 32 * g + lane;
          const bool valid = slot < 2 * nu;
          const int sl = valid ? slot : 0;
          const int bound = sl >= nu;
          const int m = lU[sl - bound * nu];
          const float sg = bound ? -1.0f : 1.0f, sg2 = 2.0f * sg;
          const float* s = sS + (bound * h + m) * ss;
          const float a1s = n_a1[m] * sg, a2 = n_a2[m];
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
              const int4 nx = k + 1 < off_end ? __ldg(R.pairs + k + 1) : pr;
              switch (pr.w) {
                BERN_CONV_SG_CASES
                default: break;
              }
              pr = nx;
            }
          }
          if (has_diag) {
            const int4 pr = __ldg(R.pairs + off_end);
            switch (pr.z & 15) {
              BERN_DIAG_SG_CASES
              default: break;
            }
          }
          float rem = 0.0f;
          const int col = n_col[m];
          float* tB = bound ? tL : tU;
          const int* rk = R.out_ranks + hd.z;
          const int el0 = hd.z - e_b;
#pragma unroll
          for (int c = 0; c < 2 * kRowLen - 1; ++c) {
            if (c >= Lout) break;
            const float lin = c < in_len ? s[in_off + c] : 0.0f;
            // sg * the value the per-step kernel forms with its own rounding
            const float vs_ = __fmaf_ru(a2, acc[c], __fmul_ru(a1s, lin));
            const int rank = __ldg(rk + c);
            if (rank == 0) {
              if (valid) s_c0[slot] = sg * vs_;
            } else if (rank < Mout) {
              if (valid) tB[(el0 + c) * vs + col] = sg * vs_;
            } else {
              rem = __fadd_ru(rem, fmaxf(vs_, 0.0f));
            }
          }
          if (A.rem_on && valid) {
            float* rp = s_rem + warp * 2 * h + slot;
            *rp = __fadd_ru(*rp, rem);
          }
        }
        __syncthreads();
        tile_to_midrad(tU, tL, E, nv, vs);
        __syncthreads();
        auto rank_of = [&](int e) { return __ldg(R.out_ranks + e); };
        if ((hn & 3) == 0)
          tile_affine<4>(A, b, sW, lV, nv, tU, tL, vs, E, e_b, rank_of, Mout);
        else
          tile_affine<1>(A, b, sW, lV, nv, tU, tL, vs, E, e_b, rank_of, Mout);
        __syncthreads();
        row_b = row_e;
      }
    } else {
      // order 1, or no unstable neuron: tiles of graded ranks 0..Mnext-1
      for (int e_b = 0; e_b < Mnext; e_b += Rcap) {
        const int E = min(Rcap, Mnext - e_b);
        for (int idx = tid; idx < E * nv; idx += kLThreads) {
          const int el = idx / nv, vi = idx - el * nv;
          const int m = lV[vi];
          const int rank = e_b + el;
          float u = 0.0f, l = 0.0f;
          if (rank < m_in) {
            const int p = __ldg(R.pos_in + rank);
            if (n_kind[m] == 1) {
              u = sS[m * ss + p];
              l = sS[(h + m) * ss + p];
            } else {
              const int Mo = T.mcount[min((int)T.deg_of[n_nt[m]], A.cap)];
              if (rank < Mo) {
                const float a1 = n_a1[m], a0 = rank == 0 ? n_a0[m] : 0.0f;
                u = __fmaf_ru(a1, sS[m * ss + p], a0);
                l = __fmaf_rd(a1, sS[(h + m) * ss + p], a0);
              }
            }
          }
          tU[el * vs + vi] = u;
          tL[el * vs + vi] = l;
        }
        __syncthreads();
        tile_to_midrad(tU, tL, E, nv, vs);
        __syncthreads();
        auto rank_of = [&](int e) { return e; };
        if ((hn & 3) == 0)
          tile_affine<4>(A, b, sW, lV, nv, tU, tL, vs, E, e_b, rank_of, Mnext);
        else
          tile_affine<1>(A, b, sW, lV, nv, tU, tL, vs, E, e_b, rank_of, Mnext);
        __syncthreads();
      }
    }

    // ---- constant terms (rank 0) of the live neurons, then rank 0 of the
    // next layer
    float* p0u = sUn;
    float* p0l = sUn + h;
    for (int slot = tid; slot < 2 * nu; slot += kLThreads) {
      const int bound = slot >= nu;
      const int m = lU[slot - bound * nu];
      const float a0 = n_a0[m], a1 = n_a1[m], a2 = n_a2[m];
      const float eta = s_eta[slot];
      float v;
      if (A.d >= 2) {
        float remt = 0.0f;
        if (A.rem_on)
          for (int w = 0; w < kLWarps; ++w) remt = __fadd_ru(remt, s_rem[w * 2 * h + slot]);
        if (bound) remt = -remt;                      // the lower remainder, rounded down
        const float lip = __fmaf_ru(2.0f * a2, __fadd_ru(1.0f, eta), fabsf(a1));
        const float c0 = s_c0[slot];
        if (!bound) {
          v = __fadd_ru(__fadd_ru(__fadd_ru(c0, a0), __fmul_ru(lip, eta)), remt);
        } else {
          v = __fsub_rd(__fadd_rd(c0, a0), __fmul_ru(lip, eta));
          v = __fadd_rd(__fsub_rd(v, n_eps[m]), remt);
        }
      } else {
        const float lip = fabsf(a1);
        const float x0 = sS[(bound * h + m) * ss];     // s at rank 0
        if (!bound) {
          v = __fadd_ru(__fmaf_ru(a1, x0, a0), __fmul_ru(lip, eta));
        } else {
          v = __fsub_rd(__fsub_rd(__fmaf_rd(a1, x0, a0), __fmul_ru(lip, eta)), n_eps[m]);
        }
      }
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
      (bound ? p0l : p0u)[n_col[m]] = v;
    }
    for (int vi = tid; vi < nv; vi += kLThreads) {
      const int m = lV[vi];
      if (n_kind[m] == 1) {
        p0u[vi] = n_nt[m] > 0 ? sS[m * ss] : 0.0f;
        p0l[vi] = n_nt[m] > 0 ? sS[(h + m) * ss] : 0.0f;
      }
    }
    __syncthreads();
    for (int mp = tid; mp < hn; mp += kLThreads) {
      float uc = A.bn[mp], lc = A.bn[mp], rad = 0.0f;
      for (int vi = 0; vi < nv; ++vi) {
        const float w = sW[lV[vi] * A.hnp + mp];
        const float u = p0u[vi], l = p0l[vi];
        const float c = __fmaf_rn(0.5f, u, 0.5f * l);
        const float rd = fmaxf(__fsub_ru(u, c), __fsub_ru(c, l));
        uc = __fmaf_ru(w, c, uc);
        lc = __fmaf_rd(w, c, lc);
        rad = __fmaf_ru(fabsf(w), rd, rad);
      }
      const int64_t o = (b * A.nx_ld) * hn + mp;
      A.nx_up[o] = __fadd_ru(uc, rad);
      A.nx_lo[o] = __fsub_rd(lc, rad);
    }
  }
}

template <int LB>
cudaError_t launch_lb(const Launch& L, const Tables& T, const LayerArgs& A, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_layer<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_layer<LB>, kLThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t blocks = std::min<int64_t>(A.n_boxes, (int64_t)device_sms(L) * per_sm);
  k_layer<LB><<<(unsigned)blocks, kLThreads, smem, L.stream>>>(T, A, T.rscale[LB], L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace

bool layer_fused_shape(int n, int h, int hn, int d, int D_pre, int order, int64_t budget, int cap,
                       LayerShape* out) {
  if (d < 1 || d > 2 || h < 1 || h > kLThreads || hn < 1 || n < 1 || n > kMaxVars) return false;
  if (D_pre < 0 || D_pre > std::min(kMaxRowDegree, row_path_max_degree(n))) return false;
  if (cap < 1 || cap > kMaxTableDegree) return false;
  int G = 0;
  // the order bern_propagate's enclosure uses (with its global-memory path):
  // grids beyond shared memory are not fused
  const int lb = effective_order(n, order, budget, &G, true);
  if (G > kEncloseGridMax || lb > kLayerMaxOrder || lb > max_enclose_order(n)) return false;
  const int64_t m_pre = num_monomials(n, D_pre);
  if (m_pre < 1) return false;
  LayerShape S;
  S.lb = lb;
  S.ss = (int)(m_pre | 1);
  S.hnp = (hn + 3) & ~3;
  const int64_t vsmax = h | 1;
  // union: the enclosure grids, the eta partial sums, the output tiles (at
  // least 32 entries at the widest live set) and the rank-0 values
  const int64_t uni = std::max<int64_t>(std::max<int64_t>((int64_t)kLWarps * G, 8LL * h),
                                        std::max<int64_t>(2LL * 32 * vsmax, 2LL * h + 2));
  S.uni = (int)uni;
  S.rem_on = 2 * D_pre > cap ? 1 : 0;
  auto r4 = [](int64_t x) { return (x + 3) & ~(int64_t)3; };
  const int64_t offW = r4(2LL * h * S.ss);
  const int64_t offU = r4(offW + (int64_t)h * S.hnp);
  const int64_t offN = r4(offU + uni);
  const int64_t words = offN + 16LL * h + (S.rem_on ? 16LL * h : 0);
  const size_t bytes = (size_t)words * 4;
  if (bytes > (size_t)kLayerSmemMax) return false;
  S.offW = (int)offW;
  S.offU = (int)offU;
  S.offN = (int)offN;
  S.smem = bytes;
  if (out) *out = S;
  return true;
}

cudaError_t launch_layer(const Launch& L, const Tables& T, int64_t n_boxes, int h, int d,
                         int order, int64_t budget, int cap, const float* pre_up,
                         const float* pre_lo, int64_t pre_ld, const int32_t* pre_nt, int hn,
                         const float* Wn, const float* bn, float* nx_up, float* nx_lo,
                         int64_t nx_ld, int32_t* nx_nt, int* counter) {
  if (n_boxes == 0) return cudaSuccess;
  if (n_boxes < 0 || n_boxes > INT32_MAX || !counter) return cudaErrorInvalidValue;
  const int n = T.n;
  int D_pre = 0;   // the largest degree whose monomials fit the layer block
  while (D_pre < kMaxTableDegree && num_monomials(n, D_pre + 1) >= 0 &&
         num_monomials(n, D_pre + 1) <= pre_ld)
    ++D_pre;
  LayerShape S;
  if (!layer_fused_shape(n, h, hn, d, D_pre, order, budget, cap, &S) || D_pre > T.row_dmax ||
      S.lb > T.rscale_max || !T.rscale[S.lb])
    return cudaErrorInvalidValue;
  LayerArgs A{n, h, d, cap, hn, n_boxes, pre_up, pre_lo, pre_ld, pre_nt, Wn, bn, nx_up, nx_lo,
              nx_ld, nx_nt, counter, S.ss, S.hnp, S.offW, S.offU, S.uni, S.offN, S.rem_on,
              (int)num_monomials(n, D_pre)};
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  switch (S.lb) {
    case 0: return launch_lb<0>(L, T, A, S.smem);
    case 1: return launch_lb<1>(L, T, A, S.smem);
    case 2: return launch_lb<2>(L, T, A, S.smem);
    case 3: return launch_lb<3>(L, T, A, S.smem);
    case 4: return launch_lb<4>(L, T, A, S.smem);
    case 5: return launch_lb<5>(L, T, A, S.smem);
    case 6: return launch_lb<6>(L, T, A, S.smem);
    case 7: return launch_lb<7>(L, T, A, S.smem);
    case 8: return launch_lb<8>(L, T, A, S.smem);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bern
