// a1: the layer step of Sec. 5.2 (eqs. upper_bounds_layer / lower_bounds_layer)
//
//   pre_up_m = b_m + sum_j W+_mj up_j + W-_mj lo_j
//   pre_lo_m = b_m + sum_j W+_mj lo_j + W-_mj up_j
//
// applied coefficient-wise over the shared graded monomial prefix.  The
// upper sum is accumulated with round-up FMAs and the lower one with
// round-down FMAs, so each computed coefficient bounds the exact one from the
// correct side; with t^K >= 0 on the box that bounds the polynomial values.
//
// The kernels for layers of more than 8 neurons (tiled, persistent wide and
// short) use the midpoint-radius form of the same step: with
// c = fl((up + lo) / 2) and r >= max(up - c, c - lo) (rounded up), every
// input coefficient lies in [c - r, c + r], and for any weight w
//   w+ up + w- lo = w c + |w| r  (exactly, when c, r are exact),
//   w x <= w c + |w| r  for every x in [c - r, c + r];
// so pre_up = RU(b + sum_j w c) + RU(sum_j |w| r) and pre_lo = RD(b + sum_j
// w c) - RU(sum_j |w| r) bound the sign-split sums from the correct side
// (r exceeds (up - lo)/2 by at most an ulp of c).  This needs three FMAs per
// product and no per-product select of the operand by the sign of w.
//
// With the layer-block layout (coefficient r of neuron j of box b at
// ((b*ld + r)*h + j)) each box is a row-major [M x h_in] matrix per bound and
// the step is the product with W^T: a small GEMM per box.  In the tiled
// kernel a block computes a BM (neurons) x BR (monomials) tile of one box; K
// (= h_in) is staged through shared memory in chunks of KC, and every thread
// keeps a TM x TR register tile per bound.  Inputs beyond a neuron's term
// count are read as zero.
#include <algorithm>
#include <string>

#include "device_util.cuh"

namespace bern {

template <int BM, int BR, int TM, int TR, int KC>
__global__ void __launch_bounds__((BM / TM) * (BR / TR))
k_affine(int h_out, int h_in, const float* __restrict__ W, const float* __restrict__ bias,
         const float* __restrict__ in_up, const float* __restrict__ in_lo, int64_t in_ld,
         const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
         float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
         int* status) {
  constexpr int NT = (BM / TM) * (BR / TR);
  constexpr int TX = BM / TM;                       // threads along m
  __shared__ float sW[KC][BM];
  __shared__ float sA[KC][BM];        // |W|
  __shared__ float sU[BR][KC + 1];    // midpoints c
  __shared__ float sL[BR][KC + 1];    // radii r
  __shared__ int sMax;
  extern __shared__ int32_t sN[];                   // h_in term counts
  const int64_t b = blockIdx.x;
  const int r0 = blockIdx.y * BR;
  const int m0 = blockIdx.z * BM;
  const int tid = threadIdx.x;
  if (tid == 0) sMax = 0;
  __syncthreads();
  int mloc = 0;
  for (int j = tid; j < h_in; j += NT) {
    int v = in_nterms[b * h_in + j];
    if (v < 0 || v > in_ld) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    sN[j] = v;
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if ((tid & 31) == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (tid == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0)
    for (int m = m0 + tid; m < min(m0 + BM, h_out); m += NT) out_nterms[b * h_out + m] = M;
  if (r0 >= M) return;

  const int tm = tid % TX, tr = tid / TX;
  float uc[TM][TR], lc[TM][TR], rad[TM][TR];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int k = 0; k < TR; ++k) {
      const int m = m0 + tm * TM + i, r = r0 + tr * TR + k;
      const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
      uc[i][k] = b0;
      lc[i][k] = b0;
      rad[i][k] = 0.0f;
    }
  const float* gU = in_up + (b * in_ld) * h_in;
  const float* gL = in_lo + (b * in_ld) * h_in;
  for (int j0 = 0; j0 < h_in; j0 += KC) {
    // stage W[m0.., j0..] transposed (and |W|), and the midpoints and radii
    // of the input rows r0.. of columns j0..
    for (int idx = tid; idx < KC * BM; idx += NT) {
      const int mm = idx % BM, jj = idx / BM;
      const int m = m0 + mm, j = j0 + jj;
      const float w = (m < h_out && j < h_in) ? W[(int64_t)m * h_in + j] : 0.0f;
      sW[jj][mm] = w;
      sA[jj][mm] = fabsf(w);
    }
    for (int idx = tid; idx < KC * BR; idx += NT) {
      const int jj = idx % KC, rr = idx / KC;
      const int j = j0 + jj, r = r0 + rr;
      float c = 0.0f, rd = 0.0f;
      if (j < h_in && r < sN[j]) {
        const float u = gU[(int64_t)r * h_in + j];
        const float l = gL[(int64_t)r * h_in + j];
        c = __fmaf_rn(0.5f, u, 0.5f * l);
        rd = fmaxf(__fsub_ru(u, c), __fsub_ru(c, l));
      }
      sU[rr][jj] = c;
      sL[rr][jj] = rd;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < KC; ++jj) {
      float w[TM], a[TM], c[TR], rd[TR];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        w[i] = sW[jj][tm * TM + i];
        a[i] = sA[jj][tm * TM + i];
      }
#pragma unroll
      for (int k = 0; k < TR; ++k) {
        c[k] = sU[tr * TR + k][jj];
        rd[k] = sL[tr * TR + k][jj];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int k = 0; k < TR; ++k) {
          uc[i][k] = __fmaf_ru(w[i], c[k], uc[i][k]);
          lc[i][k] = __fmaf_rd(w[i], c[k], lc[i][k]);
          rad[i][k] = __fmaf_ru(a[i], rd[k], rad[i][k]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TR; ++k) {
    const int r = r0 + tr * TR + k;
    if (r >= M) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tm * TM + i;
      if (m < h_out) {
        const int64_t o = (b * out_ld + r) * h_out + m;
        out_up[o] = __fadd_ru(uc[i][k], rad[i][k]);
        out_lo[o] = __fsub_rd(lc[i][k], rad[i][k]);
      }
    }
  }
}

// Persistent, register-blocked form for the wide layers: a block of four
// warps keeps W (h_in x h_out, k-major, neurons padded to 64) in shared
// memory for the whole launch and walks boxes; per box it stages 64-row tiles
// of the input as (midpoint, radius) pairs, and every thread accumulates an
// 8 (neurons) x 4 (rows) tile of the three sums per 64-neuron slice: neurons
// 4 tm .. 4 tm + 3 and 32 + 4 tm .. 32 + 4 tm + 3, so the eight lanes of a
// row read each half of the slice's weights as one contiguous 128-byte float4
// load; 4 pairs are read as float2 per input j, and |w| is taken in the
// radius FMA itself.  The staging issues kWBatch loads of each bound per
// thread before converting any.  A warp covers 16 rows of the tile and skips
// the tile when all of them are at or past the box's term count.  With a
// ScreenOut it also screens the box's output items (R21): every thread sums
// max(0, upper) and min(0, lower) of its output coefficients past the first
// (rounding up, resp. down), the four lanes of a warp that share neurons
// combine theirs, each warp adds its sum into its own shared row, and after
// the box the rows are added to the constant coefficient in warp order.
constexpr int kWThreads = 128;
constexpr int kWBatch = 8;

template <int TR, int MINB, bool SCREEN>
__global__ void __launch_bounds__(kWThreads, MINB)
k_affine_wide(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
              const float* __restrict__ bias, const float* __restrict__ in_up,
              const float* __restrict__ in_lo, int64_t in_ld,
              const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
              float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
              ScreenOut so, int* status) {
  constexpr int ROWS = 16 * TR;                      // rows per tile
  extern __shared__ float4 smem4[];
  const int hp = (h_out + 63) & ~63;                 // neurons padded to 64
  float* sW = reinterpret_cast<float*>(smem4);       // [h_in][hp]
  float2* sCR = reinterpret_cast<float2*>(sW + (size_t)h_in * hp);   // [ROWS][h_in + 1]
  int* sN = reinterpret_cast<int*>(sCR + (size_t)ROWS * (h_in + 1));   // [h_in]
  // screen partials: per warp and neuron the directed sums of max(0, upper)
  // and min(0, lower) over the warp's rows past the first, and row 0 itself
  float* sScr = reinterpret_cast<float*>(sN + h_in);   // [4][2][hp]
  float* sC0 = sScr + 8 * hp;                          // [2][hp]
  constexpr bool screen = SCREEN;
  __shared__ int sMax;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int idx = tid; idx < h_in * hp; idx += kWThreads) {
    const int j = idx / hp, m = idx - j * hp;
    sW[idx] = m < h_out ? W[(int64_t)m * h_in + j] : 0.0f;
  }
  const int tm = tid & 7, tr = tid >> 3;             // 8 x 16 threads
  const int ldx = h_in + 1;
  const int step_r = kWThreads / h_in, step_j = kWThreads - step_r * h_in;
  const bool vec_out =
      (h_out & 3) == 0 &&
      ((reinterpret_cast<uintptr_t>(out_up) | reinterpret_cast<uintptr_t>(out_lo)) & 15) == 0;
  for (int64_t b = blockIdx.x; b < n_boxes; b += gridDim.x) {
    if (tid == 0) sMax = 0;
    __syncthreads();                                 // also: W staged, previous box done
    int mloc = 0;
    for (int j = tid; j < h_in; j += kWThreads) {
      int v = in_nterms[b * h_in + j];
      if (v < 0 || v > in_ld) {
        atomicOr(status, kStatusInvalid);
        v = 0;
      }
      sN[j] = v;
      mloc = max(mloc, v);
    }
    mloc = warp_imax(mloc);
    if ((tid & 31) == 0) atomicMax(&sMax, mloc);
    __syncthreads();
    const int M = max(1, sMax);
    if (M > out_ld) {
      if (tid == 0) atomicOr(status, kStatusCapacity);
      continue;
    }
    for (int m = tid; m < h_out; m += kWThreads) out_nterms[b * h_out + m] = M;
    if (screen)
      for (int x = tid; x < 8 * hp; x += kWThreads) sScr[x] = 0.0f;
    const float* gU = in_up + (b * in_ld) * h_in;
    const float* gL = in_lo + (b * in_ld) * h_in;
    for (int r0 = 0; r0 < M; r0 += ROWS) {
      __syncthreads();                               // the previous tile is consumed
      // element idx = rr * h_in + j of the tile; (rr, j) advance by
      // (step_r, step_j) per kWThreads elements
      int rr = tid / h_in, j = tid - (tid / h_in) * h_in;
      for (int idx = tid; idx < ROWS * h_in; idx += kWThreads * kWBatch) {
        float u[kWBatch], l[kWBatch];
        int at[kWBatch];
#pragma unroll
        for (int q = 0; q < kWBatch; ++q) {
          const bool in = idx + q * kWThreads < ROWS * h_in;
          const int r = r0 + rr;
          const bool live = in && r < sN[j];         // sN[j] <= M <= in_ld
          u[q] = live ? gU[(int64_t)r * h_in + j] : 0.0f;
          l[q] = live ? gL[(int64_t)r * h_in + j] : 0.0f;
          at[q] = in ? rr * ldx + j : -1;
          rr += step_r;
          j += step_j;
          if (j >= h_in) {
            j -= h_in;
            ++rr;
          }
        }
#pragma unroll
        for (int q = 0; q < kWBatch; ++q) {
          const float c = __fmaf_rn(0.5f, u[q], 0.5f * l[q]);
          const float rd = fmaxf(__fsub_ru(u[q], c), __fsub_ru(c, l[q]));
          if (at[q] >= 0) sCR[at[q]] = make_float2(c, rd);
        }
      }
      __syncthreads();
      if (r0 + warp * 4 * TR >= M) continue;         // warp-uniform; no barrier follows
      for (int m0 = 0; m0 < h_out; m0 += 64) {
        float uc[TR][8], lc[TR][8], rad[TR][8];
#pragma unroll
        for (int k = 0; k < TR; ++k)
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? 4 * tm + i : 28 + 4 * tm + i), r = r0 + tr * TR + k;
            const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
            uc[k][i] = b0;
            lc[k][i] = b0;
            rad[k][i] = 0.0f;
          }
        const float* pw = sW + m0 + tm * 4;
        const float2* pcr = sCR + (tr * TR) * ldx;
#pragma unroll 2
        for (int j = 0; j < h_in; ++j) {
          float2 cr[TR];
#pragma unroll
          for (int k = 0; k < TR; ++k) cr[k] = pcr[k * ldx + j];
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const float4 w4 = *reinterpret_cast<const float4*>(pw + (size_t)j * hp + 32 * half);
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int k = 0; k < TR; ++k)
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int ii = 4 * half + i;
                uc[k][ii] = __fmaf_ru(w[i], cr[k].x, uc[k][ii]);
                lc[k][ii] = __fmaf_rd(w[i], cr[k].x, lc[k][ii]);
                rad[k][ii] = __fmaf_ru(fabsf(w[i]), cr[k].y, rad[k][ii]);
              }
          }
        }
#pragma unroll
        for (int k = 0; k < TR; ++k) {
          const int r = r0 + tr * TR + k;
          const bool valid = r < M;
          float vu[8], vl[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            vu[i] = __fadd_ru(uc[k][i], rad[k][i]);
            vl[i] = __fsub_rd(lc[k][i], rad[k][i]);
          }
          if (valid) {
            const int64_t o = (b * out_ld + r) * h_out + m0;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const int mb = m0 + 32 * half + 4 * tm;
              const int64_t oh = o + 32 * half + 4 * tm;
              const float* pu = vu + 4 * half;
              const float* pl = vl + 4 * half;
              if (vec_out && mb + 4 <= h_out) {
                *reinterpret_cast<float4*>(out_up + oh) = make_float4(pu[0], pu[1], pu[2], pu[3]);
                *reinterpret_cast<float4*>(out_lo + oh) = make_float4(pl[0], pl[1], pl[2], pl[3]);
              } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (mb + i < h_out) {
                    out_up[oh + i] = pu[i];
                    out_lo[oh + i] = pl[i];
                  }
              }
            }
          }
          if (screen) {   // warp-uniform (every lane runs every k)
            if (valid && r == 0) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int m = m0 + (i < 4 ? 4 * tm + i : 28 + 4 * tm + i);
                sC0[m] = vu[i];
                sC0[hp + m] = vl[i];
              }
            }
            // this row's one-sided parts, combined over the four lanes of the
            // warp that share neurons (lane, lane ^ 8, ^ 16, ^ 24), then added
            // into the warp's own shared row
            const bool part = valid && r > 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float cu = part ? fmaxf(vu[i], 0.0f) : 0.0f;
              float cl = part ? fminf(vl[i], 0.0f) : 0.0f;
              cu = __fadd_ru(cu, __shfl_xor_sync(0xffffffffu, cu, 8));
              cl = __fadd_rd(cl, __shfl_xor_sync(0xffffffffu, cl, 8));
              cu = __fadd_ru(cu, __shfl_xor_sync(0xffffffffu, cu, 16));
              cl = __fadd_rd(cl, __shfl_xor_sync(0xffffffffu, cl, 16));
              if ((tid & 31) < 8) {
                const int m = m0 + (i < 4 ? 4 * tm + i : 28 + 4 * tm + i);
                float* ps = sScr + (warp * 2) * hp + m;
                ps[0] = __fadd_ru(ps[0], cu);
                ps[hp] = __fadd_rd(ps[hp], cl);
              }
            }
          }
        }
      }
    }
    if (screen) {
      // the box's items: row 0 plus the warps' partials in warp order; the
      // stable ones get their case and interval, the others join the list
      __syncthreads();
      const int lane = tid & 31;
      for (int m0 = 0; m0 < h_out; m0 += kWThreads) {
        const int m = m0 + tid;
        bool need = false;
        if (m < h_out) {
          float u = sC0[m], l = sC0[hp + m];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            u = __fadd_ru(u, sScr[(w * 2) * hp + m]);
            l = __fadd_rd(l, sScr[(w * 2 + 1) * hp + m]);
          }
          const int64_t it = b * h_out + m;
          if (!(isfinite(l) && isfinite(u)) || (u > 0.0f && l < 0.0f)) {
            need = true;
          } else {
            so.kind[it] = u <= 0.0f ? 0 : 1;
            so.lo[it] = l;
            so.hi[it] = u;
          }
        }
        const unsigned msk = __ballot_sync(0xffffffffu, need);
        int at = 0;
        if (lane == 0 && msk) at = atomicAdd(so.count, __popc(msk));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (need) so.list[at + __popc(msk & ((1u << lane) - 1u))] = (int)(b * h_out + m);
      }
    }
  }
}

// Short polynomials (at most 16 monomial rows per box) in wide layers: the
// same register tiles as k_affine_wide, but each warp takes a whole box (its
// 16 rows x 64 neurons per slice), so a block of four warps works on four
// boxes at a time with only warp-level synchronisation after W is staged.
constexpr int kSRows = 16;

__global__ void __launch_bounds__(kWThreads, 4)
k_affine_short(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
               const float* __restrict__ bias, const float* __restrict__ in_up,
               const float* __restrict__ in_lo, int64_t in_ld,
               const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
               float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
               int* status) {
  extern __shared__ float4 smem4[];
  const int hp = (h_out + 63) & ~63;
  const int ldx = h_in + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sW = reinterpret_cast<float*>(smem4);                        // [h_in][hp]
  float2* sCR = reinterpret_cast<float2*>(sW + (size_t)h_in * hp) +
                (size_t)warp * kSRows * ldx;                          // [kSRows][ldx] per warp
  int* sN = reinterpret_cast<int*>(reinterpret_cast<float2*>(sW + (size_t)h_in * hp) +
                                   (size_t)4 * kSRows * ldx) +
            warp * h_in;                                              // [h_in] per warp
  for (int idx = threadIdx.x; idx < h_in * hp; idx += kWThreads) {
    const int j = idx / hp, m = idx - j * hp;
    sW[idx] = m < h_out ? W[(int64_t)m * h_in + j] : 0.0f;
  }
  __syncthreads();
  const int tm = lane & 7, tr = lane >> 3;           // 8 x 4 lanes
  const int step_r = 32 / h_in, step_j = 32 - step_r * h_in;
  const bool vec_out =
      (h_out & 3) == 0 &&
      ((reinterpret_cast<uintptr_t>(out_up) | reinterpret_cast<uintptr_t>(out_lo)) & 15) == 0;
  for (int64_t b = (int64_t)blockIdx.x * 4 + warp; b < n_boxes; b += (int64_t)gridDim.x * 4) {
    int mloc = 0;
    for (int j = lane; j < h_in; j += 32) {
      int v = in_nterms[b * h_in + j];
      if (v < 0 || v > in_ld) {
        atomicOr(status, kStatusInvalid);
        v = 0;
      }
      sN[j] = v;
      mloc = max(mloc, v);
    }
    const int M = max(1, warp_imax(mloc));
    if (M > out_ld || M > kSRows) {
      if (lane == 0) atomicOr(status, kStatusCapacity);
      __syncwarp();
      continue;
    }
    for (int m = lane; m < h_out; m += 32) out_nterms[b * h_out + m] = M;
    __syncwarp();                                    // sN visible to the warp
    const float* gU = in_up + (b * in_ld) * h_in;
    const float* gL = in_lo + (b * in_ld) * h_in;
    int rr = lane / h_in, j = lane - (lane / h_in) * h_in;
    for (int idx = lane; idx < M * h_in; idx += 32 * kWBatch) {
      float u[kWBatch], l[kWBatch];
      int at[kWBatch];
#pragma unroll
      for (int q = 0; q < kWBatch; ++q) {
        const bool in = idx + q * 32 < M * h_in;
        const bool live = in && rr < sN[j];
        u[q] = live ? gU[(int64_t)rr * h_in + j] : 0.0f;
        l[q] = live ? gL[(int64_t)rr * h_in + j] : 0.0f;
        at[q] = in ? rr * ldx + j : -1;
        rr += step_r;
        j += step_j;
        if (j >= h_in) {
          j -= h_in;
          ++rr;
        }
      }
#pragma unroll
      for (int q = 0; q < kWBatch; ++q) {
        const float c = __fmaf_rn(0.5f, u[q], 0.5f * l[q]);
        const float rd = fmaxf(__fsub_ru(u[q], c), __fsub_ru(c, l[q]));
        if (at[q] >= 0) sCR[at[q]] = make_float2(c, rd);
      }
    }
    __syncwarp();
    if (tr * 4 < M) {
      for (int m0 = 0; m0 < h_out; m0 += 64) {
        float uc[4][8], lc[4][8], rad[4][8];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? 4 * tm + i : 28 + 4 * tm + i), r = tr * 4 + k;
            const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
            uc[k][i] = b0;
            lc[k][i] = b0;
            rad[k][i] = 0.0f;
          }
        const float* pw = sW + m0 + tm * 4;
        const float2* pcr = sCR + (tr * 4) * ldx;
#pragma unroll 2
        for (int jj = 0; jj < h_in; ++jj) {
          float2 cr[4];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            cr[k] = tr * 4 + k < M ? pcr[k * ldx + jj] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const float4 w4 = *reinterpret_cast<const float4*>(pw + (size_t)jj * hp + 32 * half);
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int ii = 4 * half + i;
                uc[k][ii] = __fmaf_ru(w[i], cr[k].x, uc[k][ii]);
                lc[k][ii] = __fmaf_rd(w[i], cr[k].x, lc[k][ii]);
                rad[k][ii] = __fmaf_ru(fabsf(w[i]), cr[k].y, rad[k][ii]);
              }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = tr * 4 + k;
          if (r >= M) continue;
          float vu[8], vl[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            vu[i] = __fadd_ru(uc[k][i], rad[k][i]);
            vl[i] = __fsub_rd(lc[k][i], rad[k][i]);
          }
          const int64_t o = (b * out_ld + r) * h_out + m0;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int mb = m0 + 32 * half + 4 * tm;
            const int64_t oh = o + 32 * half + 4 * tm;
            const float* pu = vu + 4 * half;
            const float* pl = vl + 4 * half;
            if (vec_out && mb + 4 <= h_out) {
              *reinterpret_cast<float4*>(out_up + oh) = make_float4(pu[0], pu[1], pu[2], pu[3]);
              *reinterpret_cast<float4*>(out_lo + oh) = make_float4(pl[0], pl[1], pl[2], pl[3]);
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (mb + i < h_out) {
                  out_up[oh + i] = pu[i];
                  out_lo[oh + i] = pl[i];
                }
            }
          }
        }
      }
    }
    __syncwarp();                                    // sCR and sN consumed
  }
}

static size_t short_smem(int h_out, int h_in) {
  const size_t hp = (size_t)((h_out + 63) & ~63);
  return hp * h_in * sizeof(float) + (size_t)4 * kSRows * (h_in + 1) * sizeof(float2) +
         (size_t)4 * h_in * sizeof(int);
}

static size_t wide_smem(int h_out, int h_in, int rows) {
  const size_t hp = (size_t)((h_out + 63) & ~63);
  return hp * h_in * sizeof(float) + (size_t)rows * (h_in + 1) * sizeof(float2) +
         (size_t)h_in * sizeof(int) + 10 * hp * sizeof(float);   // + the screen partials
}

// Narrow output layers (h_out <= 4, e.g. a network's output): one thread per
// (box, monomial row) reads its whole input row (contiguous over j) and
// keeps the HO outputs of both bounds in registers; no staging is needed.
template <int HO>
__global__ void __launch_bounds__(256)
k_affine_narrow(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
                const float* __restrict__ bias, const float* __restrict__ in_up,
                const float* __restrict__ in_lo, int64_t in_ld,
                const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
                float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
                int* status) {
  extern __shared__ float sW[];                      // h_out x h_in, then h_in counts
  int32_t* sN = reinterpret_cast<int32_t*>(sW + HO * h_in);
  __shared__ int sMax;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) sMax = 0;
  for (int i = threadIdx.x; i < HO * h_in; i += blockDim.x) {
    const int m = i / h_in;
    sW[i] = m < h_out ? W[i] : 0.0f;
  }
  __syncthreads();
  int mloc = 0;
  for (int j = threadIdx.x; j < h_in; j += blockDim.x) {
    int v = in_nterms[b * h_in + j];
    if (v < 0 || v > in_ld) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    sN[j] = v;
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if ((threadIdx.x & 31) == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (threadIdx.x == 0 && blockIdx.y == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0 && threadIdx.x < h_out) out_nterms[b * h_out + threadIdx.x] = M;
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= M) return;
  float up[HO], lo[HO];
#pragma unroll
  for (int m = 0; m < HO; ++m) {
    const float b0 = (r == 0 && m < h_out) ? bias[m] : 0.0f;
    up[m] = b0;
    lo[m] = b0;
  }
  const float* pu = in_up + (b * in_ld + r) * h_in;
  const float* pl = in_lo + (b * in_ld + r) * h_in;
  auto step = [&](int j, float u, float l) {
    const bool live = r < sN[j];
    u = live ? u : 0.0f;
    l = live ? l : 0.0f;
#pragma unroll
    for (int m = 0; m < HO; ++m) {
      const float w = sW[m * h_in + j];
      const bool pos = w > 0.0f;
      up[m] = __fmaf_ru(w, pos ? u : l, up[m]);
      lo[m] = __fmaf_rd(w, pos ? l : u, lo[m]);
    }
  };
  if ((h_in & 3) == 0 && ((reinterpret_cast<uintptr_t>(pu) | reinterpret_cast<uintptr_t>(pl)) & 15) == 0) {
    // rows are 16-byte aligned: read them as float4
    const float4* pu4 = reinterpret_cast<const float4*>(pu);
    const float4* pl4 = reinterpret_cast<const float4*>(pl);
#pragma unroll 4
    for (int j4 = 0; j4 < (h_in >> 2); ++j4) {
      const float4 u = __ldg(pu4 + j4), l = __ldg(pl4 + j4);
      step(4 * j4, u.x, l.x);
      step(4 * j4 + 1, u.y, l.y);
      step(4 * j4 + 2, u.z, l.z);
      step(4 * j4 + 3, u.w, l.w);
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < h_in; ++j) step(j, __ldg(pu + j), __ldg(pl + j));
  }
#pragma unroll
  for (int m = 0; m < HO; ++m) {
    if (m < h_out) {
      const int64_t o = (b * out_ld + r) * h_out + m;
      out_up[o] = up[m];
      out_lo[o] = lo[m];
    }
  }
}

// Narrow layers (h_out <= 4), warp form: a block takes one box and 64
// monomial rows, a warp one row at a time with its lanes over the inputs j
// (coalesced row reads; each lane keeps its inputs' weights and term counts
// in registers); the per-lane partial sums are combined by a directed warp
// reduction (round-up for the upper sum, round-down for the lower one), which
// bounds the exact sum from the correct side in any order.
constexpr int kNarrowMaxJ = 8;                       // h_in <= 256

template <int HO, int JQ>
__global__ void __launch_bounds__(256)
k_affine_narrow_warp(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
                     const float* __restrict__ bias, const float* __restrict__ in_up,
                     const float* __restrict__ in_lo, int64_t in_ld,
                     const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
                     float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
                     int* status) {
  __shared__ int sMax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) sMax = 0;
  __syncthreads();
  float w[HO][JQ];
  int nt[JQ];
  int mloc = 0;
#pragma unroll
  for (int q = 0; q < JQ; ++q) {
    const int j = lane + 32 * q;
    int v = 0;
    if (j < h_in) {
      v = in_nterms[b * h_in + j];
      if (v < 0 || v > in_ld) {
        atomicOr(status, kStatusInvalid);
        v = 0;
      }
    }
    nt[q] = v;
    mloc = max(mloc, v);
#pragma unroll
    for (int m = 0; m < HO; ++m) w[m][q] = (j < h_in && m < h_out) ? W[(int64_t)m * h_in + j] : 0.0f;
  }
  mloc = warp_imax(mloc);
  if (lane == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (threadIdx.x == 0 && blockIdx.y == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0 && threadIdx.x < h_out) out_nterms[b * h_out + threadIdx.x] = M;
  const int r_end = min(M, (int)(blockIdx.y + 1) * 64);
  for (int r = blockIdx.y * 64 + warp; r < r_end; r += 8) {
    const float* pu = in_up + (b * in_ld + r) * h_in;
    const float* pl = in_lo + (b * in_ld + r) * h_in;
    float u[JQ], l[JQ];
#pragma unroll
    for (int q = 0; q < JQ; ++q) {
      const int j = lane + 32 * q;
      const bool live = j < h_in && r < nt[q];
      u[q] = live ? __ldg(pu + j) : 0.0f;
      l[q] = live ? __ldg(pl + j) : 0.0f;
    }
    float up[HO], lo[HO];
#pragma unroll
    for (int m = 0; m < HO; ++m) {
      up[m] = 0.0f;
      lo[m] = 0.0f;
#pragma unroll
      for (int q = 0; q < JQ; ++q) {
        const bool pos = w[m][q] > 0.0f;
        up[m] = __fmaf_ru(w[m][q], pos ? u[q] : l[q], up[m]);
        lo[m] = __fmaf_rd(w[m][q], pos ? l[q] : u[q], lo[m]);
      }
      up[m] = warp_dsum<true>(up[m]);
      lo[m] = warp_dsum<false>(lo[m]);
    }
    if (lane < h_out) {
      float vu = 0.0f, vl = 0.0f;
#pragma unroll
      for (int m = 0; m < HO; ++m)
        if (m == lane) {
          vu = up[m];
          vl = lo[m];
        }
      if (r == 0) {
        vu = __fadd_ru(vu, bias[lane]);
        vl = __fadd_rd(vl, bias[lane]);
      }
      const int64_t o = (b * out_ld + r) * h_out + lane;
      out_up[o] = vu;
      out_lo[o] = vl;
    }
  }
}

// Narrow layers (h_out <= 4) with h_in a multiple of 4 and 16-byte aligned
// rows, quad form: G lanes share one monomial row, each lane reading four
// consecutive inputs j as one float4, so a warp reads 32 / G whole rows per
// load; U such loads are issued before any is used.  Each lane keeps the
// weights and term counts of its four inputs in registers (and skips the
// loads of rows past all four counts); the G partial sums
// of a row are combined by a directed shuffle reduction (round-up for the
// upper sum, round-down for the lower one), which bounds the exact sum from
// the correct side in any order.  A block takes one box and kQRows rows.
constexpr int kQRows = 256;

template <int HO, int G>
__global__ void __launch_bounds__(256)
k_affine_narrow_quad(int64_t n_boxes, int h_out, int h_in, const float* __restrict__ W,
                     const float* __restrict__ bias, const float* __restrict__ in_up,
                     const float* __restrict__ in_lo, int64_t in_ld,
                     const int32_t* __restrict__ in_nterms, float* __restrict__ out_up,
                     float* __restrict__ out_lo, int64_t out_ld, int32_t* __restrict__ out_nterms,
                     int* status) {
  constexpr int R = 32 / G;                          // rows per warp load
  constexpr int U = 4;                               // loads in flight per warp
  __shared__ int sMax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = lane % G, s = lane / G;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) sMax = 0;
  __syncthreads();
  int mloc = 0;
  for (int j = threadIdx.x; j < h_in; j += blockDim.x) {
    int v = in_nterms[b * h_in + j];
    if (v < 0 || v > in_ld) {
      atomicOr(status, kStatusInvalid);
      v = 0;
    }
    mloc = max(mloc, v);
  }
  mloc = warp_imax(mloc);
  if (lane == 0) atomicMax(&sMax, mloc);
  __syncthreads();
  const int M = max(1, sMax);
  if (M > out_ld) {
    if (threadIdx.x == 0 && blockIdx.y == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  if (blockIdx.y == 0 && threadIdx.x < h_out) out_nterms[b * h_out + threadIdx.x] = M;
  const bool qlive = 4 * q < h_in;
  float w[HO][4];
  int nt[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = 4 * q + i;
    int v = qlive ? in_nterms[b * h_in + j] : 0;
    nt[i] = (v < 0 || v > in_ld) ? 0 : v;
#pragma unroll
    for (int m = 0; m < HO; ++m) w[m][i] = (qlive && m < h_out) ? W[(int64_t)m * h_in + j] : 0.0f;
  }
  const float4* pu = reinterpret_cast<const float4*>(in_up + (b * in_ld) * h_in) + q;
  const float4* pl = reinterpret_cast<const float4*>(in_lo + (b * in_ld) * h_in) + q;
  const int h4 = h_in >> 2;
  const int ntq = max(max(nt[0], nt[1]), max(nt[2], nt[3]));   // rows this quad holds
  const int r_end = min(M, (int)(blockIdx.y + 1) * kQRows);
  for (int r0 = blockIdx.y * kQRows + warp * R * U; r0 < r_end; r0 += 8 * R * U) {
    float4 u[U], l[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int r = r0 + k * R + s;
      if (qlive && r < r_end && r < ntq) {
        u[k] = __ldg(pu + (int64_t)r * h4);
        l[k] = __ldg(pl + (int64_t)r * h4);
      } else {
        u[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        l[k] = u[k];
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int r = r0 + k * R + s;
      const float uu[4] = {r < nt[0] ? u[k].x : 0.0f, r < nt[1] ? u[k].y : 0.0f,
                           r < nt[2] ? u[k].z : 0.0f, r < nt[3] ? u[k].w : 0.0f};
      const float ll[4] = {r < nt[0] ? l[k].x : 0.0f, r < nt[1] ? l[k].y : 0.0f,
                           r < nt[2] ? l[k].z : 0.0f, r < nt[3] ? l[k].w : 0.0f};
      float up[HO], lo[HO];
#pragma unroll
      for (int m = 0; m < HO; ++m) {
        up[m] = 0.0f;
        lo[m] = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool pos = w[m][i] > 0.0f;
          up[m] = __fmaf_ru(w[m][i], pos ? uu[i] : ll[i], up[m]);
          lo[m] = __fmaf_rd(w[m][i], pos ? ll[i] : uu[i], lo[m]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
          up[m] = __fadd_ru(up[m], __shfl_xor_sync(0xffffffffu, up[m], o));
          lo[m] = __fadd_rd(lo[m], __shfl_xor_sync(0xffffffffu, lo[m], o));
        }
      }
      if (q == 0 && r < r_end) {
#pragma unroll
        for (int m = 0; m < HO; ++m) {
          if (m < h_out) {
            float vu = up[m], vl = lo[m];
            if (r == 0) {
              vu = __fadd_ru(vu, bias[m]);
              vl = __fadd_rd(vl, bias[m]);
            }
            const int64_t o = (b * out_ld + r) * h_out + m;
            out_up[o] = vu;
            out_lo[o] = vl;
          }
        }
      }
    }
  }
}

template <int BM, int BR, int TM, int TR, int KC>
static cudaError_t launch_cfg(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                              const float* W, const float* b, const float* in_up,
                              const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                              float* out_up, float* out_lo, int64_t out_ld,
                              int32_t* out_nterms) {
  // r tiles cover the largest possible term count (in_ld); tiles past a box's
  // actual count exit after the count is known
  const int64_t rt = (std::max<int64_t>(1, std::min(in_ld, out_ld)) + BR - 1) / BR;
  dim3 grid((unsigned)n_boxes, (unsigned)rt, (unsigned)((h_out + BM - 1) / BM));
  const size_t smem = (size_t)h_in * sizeof(int32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_affine<BM, BR, TM, TR, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_affine<BM, BR, TM, TR, KC><<<grid, (BM / TM) * (BR / TR), smem, L.stream>>>(
      h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld, out_nterms,
      L.status);
  ++*L.launches;
  return cudaGetLastError();
}

cudaError_t launch_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                          const float* W, const float* b, const float* in_up,
                          const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                          float* out_up, float* out_lo, int64_t out_ld,
                          int32_t* out_nterms, const ScreenOut* screen, bool* screened) {
  if (screened) *screened = false;
  if (n_boxes == 0) return cudaSuccess;
  if (n_boxes > 0x7fffffff || (std::min(in_ld, out_ld) + 15) / 16 > 65535)
    return cudaErrorInvalidValue;
  const bool few_rows = std::min(in_ld, out_ld) <= 16;     // short polynomials: short tiles
  if (h_out >= 32) {
    // wide layers: autotuned among the persistent register-blocked kernel with
    // 4-row (0), 2-row (2, the default for longer polynomials) or 1-row (3)
    // thread tiles, when its weights fit shared memory, block tiles (1), and
    // for short polynomials a warp per box (4, their default)
    const std::string key = "affine/" + std::to_string(h_out) + "/" + std::to_string(h_in) +
                            "/" + std::to_string(in_ld) + "/" + std::to_string(n_boxes);
    const bool wide_ok = wide_smem(h_out, h_in, 64) <= 200 * 1024;
    const size_t ssmem = short_smem(h_out, h_in);
    const bool short_ok = few_rows && ssmem <= 200 * 1024;
    int v = tune_variant(L, "affine", key, short_ok ? 4 : (wide_ok ? 2 : 1));
    if (v == 4 && !short_ok) v = wide_ok ? 2 : 1;
    if (v != 1 && v != 4 && !wide_ok) v = short_ok ? 4 : 1;
    TuneTimer tt;
    tune_begin(L, "affine", tt);
    cudaError_t e;
    if (v == 0 || v == 2 || v == 3) {
      const int rows = v == 0 ? 64 : (v == 2 ? 32 : 16);
      const size_t wsmem = wide_smem(h_out, h_in, rows);
      auto kern = screen ? (v == 0 ? k_affine_wide<4, 4, true>
                                   : (v == 2 ? k_affine_wide<2, 6, true> : k_affine_wide<1, 8, true>))
                         : (v == 0 ? k_affine_wide<4, 4, false>
                                   : (v == 2 ? k_affine_wide<2, 6, false>
                                             : k_affine_wide<1, 8, false>));
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
      if (e != cudaSuccess) return e;
      const int max_sm = v == 0 ? 4 : (v == 2 ? 6 : 8);
      int per_sm = (int)std::min<size_t>(max_sm, (220 * 1024) / (wsmem + 1024));
      if (per_sm < 1) per_sm = 1;
      const int64_t blocks = std::min<int64_t>(n_boxes, device_sms(L) * per_sm);
      kern<<<(unsigned)blocks, kWThreads, wsmem, L.stream>>>(
          n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld,
          out_nterms, screen ? *screen : ScreenOut{}, L.status);
      ++*L.launches;
      e = cudaGetLastError();
      if (screen && screened) *screened = true;
    } else if (v == 4) {
      e = cudaFuncSetAttribute(k_affine_short, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ssmem);
      if (e != cudaSuccess) return e;
      const int per_sm = ssmem <= 54 * 1024 ? 4 : (ssmem <= 72 * 1024 ? 3 : (ssmem <= 110 * 1024 ? 2 : 1));
      const int64_t blocks = std::min<int64_t>((n_boxes + 3) / 4, device_sms(L) * per_sm);
      k_affine_short<<<(unsigned)blocks, kWThreads, ssmem, L.stream>>>(
          n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld,
          out_nterms, L.status);
      ++*L.launches;
      e = cudaGetLastError();
    } else if (few_rows) {
      e = launch_cfg<64, 16, 4, 1, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                       in_nterms, out_up, out_lo, out_ld, out_nterms);
    } else {
      e = launch_cfg<64, 32, 4, 2, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                       in_nterms, out_up, out_lo, out_ld, out_nterms);
    }
    tune_end(L, "affine", key, tt);
    return e;
  }
  if (h_out > 8 && few_rows)
    return launch_cfg<16, 16, 2, 1, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  if (h_out > 8)
    return launch_cfg<16, 64, 2, 4, 32>(L, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                        in_nterms, out_up, out_lo, out_ld, out_nterms);
  // narrow outputs (h_out <= 4, h_in <= 128 a multiple of 4, aligned rows):
  // lanes over float4 quads of a row
  if (h_out <= 4 && (h_in & 3) == 0 && h_in <= 128 &&
      ((reinterpret_cast<uintptr_t>(in_up) | reinterpret_cast<uintptr_t>(in_lo)) & 15) == 0) {
    const int64_t rows = std::max<int64_t>(1, std::min(in_ld, out_ld));
    if ((rows + kQRows - 1) / kQRows > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)n_boxes, (unsigned)((rows + kQRows - 1) / kQRows));
    const int q4 = h_in >> 2;
    const int g = q4 <= 4 ? 4 : (q4 <= 8 ? 8 : (q4 <= 16 ? 16 : 32));
#define BERN_NQ(HO, G)                                                                        \
  if ((HO == 1) == (h_out == 1) && g == G)                                                    \
    k_affine_narrow_quad<HO, G><<<grid, 256, 0, L.stream>>>(                                  \
        n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld,   \
        out_nterms, L.status);
    BERN_NQ(1, 4) BERN_NQ(1, 8) BERN_NQ(1, 16) BERN_NQ(1, 32)
    BERN_NQ(4, 4) BERN_NQ(4, 8) BERN_NQ(4, 16) BERN_NQ(4, 32)
#undef BERN_NQ
    ++*L.launches;
    return cudaGetLastError();
  }
  // narrow outputs (h_out <= 4, h_in <= 256): a warp per monomial row
  if (h_out <= 4 && h_in <= 32 * kNarrowMaxJ) {
    const int64_t rows = std::max<int64_t>(1, std::min(in_ld, out_ld));
    if ((rows + 63) / 64 > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)n_boxes, (unsigned)((rows + 63) / 64));
    const int jq = h_in <= 32 ? 1 : (h_in <= 64 ? 2 : (h_in <= 128 ? 4 : 8));
#define BERN_NW(HO, JQ)                                                                       \
  if ((HO == 1) == (h_out == 1) && jq == JQ)                                                  \
    k_affine_narrow_warp<HO, JQ><<<grid, 256, 0, L.stream>>>(                                 \
        n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms, out_up, out_lo, out_ld,   \
        out_nterms, L.status);
    BERN_NW(1, 1) BERN_NW(1, 2) BERN_NW(1, 4) BERN_NW(1, 8)
    BERN_NW(4, 1) BERN_NW(4, 2) BERN_NW(4, 4) BERN_NW(4, 8)
#undef BERN_NW
    ++*L.launches;
    return cudaGetLastError();
  }
  // narrow outputs (h_out <= 8): a thread per monomial row, HO >= h_out
  const int HO = h_out == 1 ? 1 : (h_out <= 4 ? 4 : 8);
  const size_t smem = (size_t)HO * h_in * sizeof(float) + (size_t)h_in * sizeof(int32_t);
  const int64_t rows = std::max<int64_t>(1, std::min(in_ld, out_ld));
  if (smem > 200 * 1024 || (rows + 127) / 128 > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)n_boxes, (unsigned)((rows + 127) / 128));
  cudaError_t e = cudaSuccess;
#define BERN_NARROW(X)                                                                        \
  if (HO == X) {                                                                              \
    if (smem > 48 * 1024)                                                                     \
      e = cudaFuncSetAttribute(k_affine_narrow<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)smem);                                                    \
    if (e == cudaSuccess)                                                                     \
      k_affine_narrow<X><<<grid, 128, smem, L.stream>>>(n_boxes, h_out, h_in, W, b, in_up,    \
                                                        in_lo, in_ld, in_nterms, out_up,      \
                                                        out_lo, out_ld, out_nterms, L.status);\
  }
  BERN_NARROW(1)
  BERN_NARROW(4)
  BERN_NARROW(8)
#undef BERN_NARROW
  if (e != cudaSuccess) return e;
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
