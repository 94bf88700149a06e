// a2 for Bernstein grids larger than shared memory (Sec. 5.1 Step 1 with
// Def. 2, the full tensor-product grid of order l in every variable):
// (l+1)^n cells up to the caller's budget, e.g. 9^6 = 531,441 cells for six
// inputs at order 8.  One block per polynomial works on its own slice of a
// global workspace (resident in L2 while the block runs): the scaled
// coefficients are scattered to their grid cells, then the per-variable
// triangular transforms run from the last variable to the first, the threads
// of the block taking the lines of a pass (a line = the l+1 cells that differ
// only in one variable), with a block barrier between passes; the first
// variable's pass feeds the min/max.  The arithmetic is that of the
// shared-memory kernels (enclose_impl.cuh): the same reciprocal brackets,
// the same in-simplex line selection (a polynomial of total degree D <= l
// occupies the simplex of digit sums <= D, so a line whose untransformed
// prefix leaves it is skipped and no cell needs zeroing), the same
// compile-time line transforms with directed FMAs, so every coefficient is a
// one-sided bound of the exact one.  Line offsets are decoded from the line
// index in mixed radix l+1 (no line tables).
#include "enclose_impl.cuh"

namespace bern {

namespace {

constexpr int kBigThreads = 512;

template <int LB, bool UP, int NT>
__device__ float enclose_block_big(const float* __restrict__ P, int ps, int nt, int n,
                                   const Tables& T, const float2* __restrict__ rs, float* grid,
                                   float* red) {
  constexpr int R = LB + 1;
  const int tid = threadIdx.x;
  const int Dnt = prefix_degree(T, nt);
  const int Deff = Dnt < LB ? Dnt : LB;
  const int m_eff = T.mcount[Deff];
  const int32_t* __restrict__ gidx = T.gidx[LB];
  // scatter (block-strided; the remainder of terms above the order)
  float rem = 0.0f;
  for (int r = tid; r < nt; r += NT) {
    const float a = P[(int64_t)r * ps];
    if (r < m_eff) {
      const float2 sc = rs[r];
      grid[__ldg(gidx + r)] = UP ? __fmul_ru(a, a >= 0.0f ? sc.y : sc.x)
                                 : __fmul_rd(a, a >= 0.0f ? sc.x : sc.y);
    } else {
      rem = UP ? __fadd_ru(rem, fmaxf(a, 0.0f)) : __fadd_rd(rem, fminf(a, 0.0f));
    }
  }
  for (int r = nt + tid; r < m_eff; r += NT) grid[__ldg(gidx + r)] = 0.0f;
  __syncthreads();
  float best = UP ? -CUDART_INF_F : CUDART_INF_F;
  int nlines = 1;
  for (int k = 0; k < n - 1; ++k) nlines *= R;
  for (int k = n - 1; k >= 0; --k) {
    int sk = 1;
    for (int j = k + 1; j < n; ++j) sk *= R;
    for (int Ln = tid; Ln < nlines; Ln += NT) {
      // digits of the other variables, the highest variable first
      int rest = Ln, base = 0, psum = 0, pw = 1;
      for (int mm = n - 1; mm >= 0; --mm) {
        if (mm == k) {
          pw *= R;
          continue;
        }
        const int dgt = rest % R;
        rest /= R;
        base += dgt * pw;
        if (mm < k) psum += dgt;
        pw *= R;
      }
      if (psum > Deff) continue;
      const int p = Deff - psum;
      float x[R], y[R];
#pragma unroll
      for (int j = 0; j < R; ++j) x[j] = j <= p ? grid[base + j * sk] : 0.0f;
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
    __syncthreads();
  }
  // block reductions: max/min of the coefficients, directed sum of the rest
  best = UP ? warp_max(best) : warp_min(best);
  rem = warp_dsum<UP>(rem);
  const int lane = tid & 31, wid = tid >> 5;
  if (lane == 0) {
    red[wid] = best;
    red[32 + wid] = rem;
  }
  __syncthreads();
  float v = 0.0f;
  if (wid == 0) {
    constexpr int kW = NT / 32;
    float b2 = lane < kW ? red[lane] : (UP ? -CUDART_INF_F : CUDART_INF_F);
    float r2 = lane < kW ? red[32 + lane] : 0.0f;
    b2 = UP ? warp_max(b2) : warp_min(b2);
    r2 = warp_dsum<UP>(r2);
    v = dadd<UP>(b2, r2);
  }
  __syncthreads();   // red and the grid slice are reused by the next polynomial
  return v;
}

// Polynomials p = 2*list_index + bound of the launch's items; persistent
// blocks, each with its own workspace slice of G floats.
template <int LB>
__global__ void __launch_bounds__(kBigThreads)
k_enclose_big(Tables T, int G, const float2* __restrict__ rs, int64_t n_items, int h,
              const float* __restrict__ pre_up, const float* __restrict__ pre_lo, int64_t ld,
              const int32_t* __restrict__ nterms, float* __restrict__ lo, float* __restrict__ hi,
              const int* list, const int* count, float* ws, int* status) {
  __shared__ float red[64];
  float* grid = ws + (size_t)blockIdx.x * G;
  const int64_t n_list = list ? (int64_t)*count : n_items;
  for (int64_t p = blockIdx.x; p < 2 * n_list; p += gridDim.x) {
    const int64_t idx = p >> 1;
    const bool up = p & 1;
    const int64_t item = list ? (int64_t)list[idx] : idx;
    int nt = nterms[item];
    if (nt < 0 || nt > ld || nt > T.mexps) {
      if (threadIdx.x == 0) atomicOr(status, kStatusInvalid);
      nt = 0;
    }
    const int64_t b = item / h;
    const int64_t base = (b * ld) * h + (item - b * h);
    const float v =
        up ? enclose_block_big<LB, true, kBigThreads>(pre_up + base, h, nt, T.n, T, rs, grid, red)
           : enclose_block_big<LB, false, kBigThreads>(pre_lo + base, h, nt, T.n, T, rs, grid, red);
    if (threadIdx.x == 0) {
      (up ? hi : lo)[item] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  }
}

// The same block-level transforms on grids in shared memory, for grids that
// fit it but leave a warp-per-polynomial launch few warps per SM (e.g. 17^3
// = 4913 cells, 19.6 KB, at order 16 in three variables): one block of
// 128 or 320 threads per polynomial, as many blocks per SM as the grids and
// threads allow.
template <int LB, int NT>
__global__ void __launch_bounds__(NT)
k_enclose_blk(Tables T, const float2* __restrict__ rs, int64_t n_items, int h,
              const float* __restrict__ pre_up, const float* __restrict__ pre_lo, int64_t ld,
              const int32_t* __restrict__ nterms, float* __restrict__ lo, float* __restrict__ hi,
              const int* list, const int* count, int* status) {
  extern __shared__ float sgrid[];
  __shared__ float red[64];
  const int64_t n_list = list ? (int64_t)*count : n_items;
  for (int64_t p = blockIdx.x; p < 2 * n_list; p += gridDim.x) {
    const int64_t idx = p >> 1;
    const bool up = p & 1;
    const int64_t item = list ? (int64_t)list[idx] : idx;
    int nt = nterms[item];
    if (nt < 0 || nt > ld || nt > T.mexps) {
      if (threadIdx.x == 0) atomicOr(status, kStatusInvalid);
      nt = 0;
    }
    const int64_t b = item / h;
    const int64_t base = (b * ld) * h + (item - b * h);
    const float v =
        up ? enclose_block_big<LB, true, NT>(pre_up + base, h, nt, T.n, T, rs, sgrid, red)
           : enclose_block_big<LB, false, NT>(pre_lo + base, h, nt, T.n, T, rs, sgrid, red);
    if (threadIdx.x == 0) {
      (up ? hi : lo)[item] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  }
}

template <int LB, int NT>
cudaError_t launch_blk_nt(const Launch& L, const Tables& T, int G, int64_t n_items, int h,
                          const float* pre_up, const float* pre_lo, int64_t ld,
                          const int32_t* nterms, float* lo, float* hi, const int* list,
                          const int* count) {
  const size_t smem = (size_t)G * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_enclose_blk<LB, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int by_smem = (int)((220 * 1024) / (smem + 1024)), by_threads = 2048 / NT;
  const int per_sm = std::max(1, std::min(16, std::min(by_smem, by_threads)));
  const int64_t blocks = std::min<int64_t>((int64_t)device_sms(L) * per_sm, 2 * n_items);
  k_enclose_blk<LB, NT><<<(unsigned)blocks, NT, smem, L.stream>>>(
      T, T.rscale[LB], n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, list, count, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// 128 threads a polynomial, or 320 (a pass over the 289 lines of a 17^3 grid
// in one round)
template <int LB>
cudaError_t launch_blk_lb(const Launch& L, const Tables& T, int G, int64_t n_items, int h,
                          const float* pre_up, const float* pre_lo, int64_t ld,
                          const int32_t* nterms, float* lo, float* hi, const int* list,
                          const int* count, bool wide) {
  return wide ? launch_blk_nt<LB, 320>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi,
                                       list, count)
              : launch_blk_nt<LB, 128>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi,
                                       list, count);
}

template <int LB>
cudaError_t launch_big_lb(const Launch& L, const Tables& T, int G, int64_t n_items, int h,
                          const float* pre_up, const float* pre_lo, int64_t ld,
                          const int32_t* nterms, float* lo, float* hi, const int* list,
                          const int* count) {
  const int64_t slices = L.ews_floats / G;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>(slices, 2LL * device_sms(L)),
                                           2 * n_items);
  if (blocks < 1) return cudaErrorInvalidValue;
  k_enclose_big<LB><<<(unsigned)blocks, kBigThreads, 0, L.stream>>>(
      T, G, T.rscale[LB], n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, list, count, L.ews,
      L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_enclose_blk(const Launch& L, const Tables& T, int lb, int G, int64_t n_items,
                               int h, const float* pre_up, const float* pre_lo, int64_t ld,
                               const int32_t* nterms, float* lo, float* hi, const int* list,
                               const int* count, bool wide) {
  if (lb > T.rscale_max || !T.rscale[lb] || !T.gidx[lb]) return cudaErrorInvalidValue;
#define BERN_BLK_CASE(X) \
  case X: return launch_blk_lb<X>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, list, \
                                  count, wide);
  switch (lb) {
    BERN_BLK_CASE(3) BERN_BLK_CASE(4) BERN_BLK_CASE(5) BERN_BLK_CASE(6) BERN_BLK_CASE(7)
    BERN_BLK_CASE(8) BERN_BLK_CASE(9) BERN_BLK_CASE(10) BERN_BLK_CASE(11) BERN_BLK_CASE(12)
    BERN_BLK_CASE(13) BERN_BLK_CASE(14) BERN_BLK_CASE(15) BERN_BLK_CASE(16)
    default: return cudaErrorInvalidValue;
  }
#undef BERN_BLK_CASE
}

size_t enclose_big_floats(int n, int order, int64_t budget, int sms) {
  int G = 0;
  effective_order(n, order, budget, &G, true);
  if (G <= kEncloseGridMax) return 0;
  const int64_t cap = kEncloseBigBytes / (4 * (int64_t)G);   // slices within the cap
  return (size_t)G * (size_t)std::max<int64_t>(1, std::min<int64_t>(cap, 2LL * sms));
}

cudaError_t launch_enclose_big(const Launch& L, const Tables& T, int lb, int G, int64_t n_items,
                               int h, const float* pre_up, const float* pre_lo, int64_t ld,
                               const int32_t* nterms, float* lo, float* hi, const int* list,
                               const int* count) {
  if (!L.ews || lb > T.rscale_max || !T.rscale[lb] || !T.gidx[lb]) return cudaErrorInvalidValue;
#define BERN_BIG_CASE(X) \
  case X: return launch_big_lb<X>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, list, count);
  switch (lb) {
    BERN_BIG_CASE(2) BERN_BIG_CASE(3) BERN_BIG_CASE(4) BERN_BIG_CASE(5) BERN_BIG_CASE(6)
    BERN_BIG_CASE(7) BERN_BIG_CASE(8) BERN_BIG_CASE(9) BERN_BIG_CASE(10) BERN_BIG_CASE(11)
    BERN_BIG_CASE(12) BERN_BIG_CASE(13) BERN_BIG_CASE(14) BERN_BIG_CASE(15) BERN_BIG_CASE(16)
    default: return cudaErrorInvalidValue;
  }
#undef BERN_BIG_CASE
}

}  // namespace bern
