// Bernstein enclosure (a2) and ReLU coefficients (a3): dispatch over the
// effective Bernstein order.  The per-order kernels are instantiated here
// (orders 0-8) and in k_enclose_hi.cu (9-16); orders above 16 use the
// runtime-order kernel below.
#include <string>

#include "enclose_impl.cuh"

namespace bern {

#define BERN_ENC_EXTERN(X)                                                                   \
  extern template cudaError_t launch_lb<X>(const Launch&, const Tables&, int, int64_t, int,  \
                                           const float*, const float*, int64_t, const int32_t*, \
                                           float*, float*, EncloseOpts);
BERN_ENC_EXTERN(9) BERN_ENC_EXTERN(10) BERN_ENC_EXTERN(11) BERN_ENC_EXTERN(12)
BERN_ENC_EXTERN(13) BERN_ENC_EXTERN(14) BERN_ENC_EXTERN(15) BERN_ENC_EXTERN(16)
#undef BERN_ENC_EXTERN

__global__ void __launch_bounds__(512)
k_enclose_generic(Tables T, int lb, int G, const float2* __restrict__ rs, int64_t n_items, int h,
                  const float* __restrict__ pre_up, const float* __restrict__ pre_lo,
                  int64_t ld, const int32_t* __restrict__ nterms, float* __restrict__ lo,
                  float* __restrict__ hi, EncloseOpts ro, int* status) {
  extern __shared__ float smem[];
  __shared__ float s_lohi[8][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_block = blockDim.x >> 6;
  const int64_t item = map_item(ro, (int64_t)blockIdx.x * per_block + (warp >> 1), n_items);
  const bool up = warp & 1;
  if (item >= 0) {
    int nt = nterms[item];
    if (nt < 0 || nt > ld || nt > T.mexps) {
      if (lane == 0) atomicOr(status, kStatusInvalid);
      nt = 0;
    }
    const int64_t b = item / h;
    const int64_t base = (b * ld) * h + (item - b * h);
    float* grid = smem + warp * G;
    const float v =
        up ? enclose_warp_generic<true>(pre_up + base, h, nt, T.n, lb, T, rs, grid)
           : enclose_warp_generic<false>(pre_lo + base, h, nt, T.n, lb, T, rs, grid);
    if (lane == 0) {
      (up ? hi : lo)[item] = v;
      s_lohi[warp >> 1][up ? 1 : 0] = v;
      if (!isfinite(v)) atomicOr(status, kStatusNonFinite);
    }
  }
  if (ro.kind == nullptr) return;
  __syncthreads();
  if (threadIdx.x < per_block) {
    const int64_t it = map_item(ro, (int64_t)blockIdx.x * per_block + threadIdx.x, n_items);
    if (it >= 0) {
      const int d = ro.degrees ? (int)ro.degrees[it] : ro.global_d;
      ro.kind[it] = (int8_t)relu_item(s_lohi[threadIdx.x][0], s_lohi[threadIdx.x][1], d,
                                      ro.coef + it * kCoefStride, ro.eps + it, status);
    }
  }
}

static cudaError_t launch_generic(const Launch& L, const Tables& T, int lb, int G,
                                  int64_t n_items, int h, const float* pre_up,
                                  const float* pre_lo, int64_t ld, const int32_t* nterms,
                                  float* lo, float* hi, EncloseOpts ro) {
  int items = (int)std::min<int64_t>(8, (192 * 1024) / (2 * (int64_t)G * 4));
  if (items < 1) items = 1;
  const size_t smem = (size_t)2 * items * G * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_enclose_generic,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((n_items + items - 1) / items);
  k_enclose_generic<<<blocks, 64 * items, smem, L.stream>>>(T, lb, G, T.rscale[lb], n_items, h,
                                                           pre_up, pre_lo, ld, nterms, lo, hi,
                                                           ro, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

// Effective Bernstein order: the requested order, lowered until the grid
// fits both the caller's budget and the grid limit (shared memory, or with
// the global-memory path BERN_MAX_BIG_GRID at orders <= 16), and the
// exact-binomial limit.  Terms above it are enclosed by coefficient
// intervals (budget rule).
int effective_order(int n, int order, int64_t budget, int* grid_out, bool big) {
  if (budget <= 0) budget = (int64_t)1 << 20;
  const int64_t gmax = big ? (int64_t)BERN_MAX_BIG_GRID : (int64_t)kEncloseGridMax;
  const int64_t lim = budget < gmax ? budget : gmax;
  int lb = order < kMaxEncloseOrder ? order : kMaxEncloseOrder;
  for (; lb > 0; --lb) {
    int64_t g = 1;
    for (int k = 0; k < n && g <= lim; ++k) g *= (lb + 1);
    if (g <= lim && (g <= kEncloseGridMax || lb <= 16)) break;
  }
  int64_t g = 1;
  for (int k = 0; k < n; ++k) g *= (lb + 1);
  *grid_out = (int)g;
  return lb;
}

// ReLU cases and coefficients of the items of a list (the enclosure of grids
// above shared memory computes lo/hi only).
__global__ void k_relu_coeffs_list(const int* __restrict__ list, const int* __restrict__ count,
                                   int64_t n_items, const float* __restrict__ lo,
                                   const float* __restrict__ hi, const uint8_t* __restrict__ degrees,
                                   int global_d, int8_t* __restrict__ kind, float* __restrict__ coef,
                                   float* __restrict__ eps, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = list ? (int64_t)*count : n_items;
  if (i >= n) return;
  const int64_t it = list ? (int64_t)list[i] : i;
  const int d = degrees ? (int)degrees[it] : global_d;
  kind[it] = (int8_t)relu_item(lo[it], hi[it], d, coef + it * kCoefStride, eps + it, status);
}

static cudaError_t launch_enclose_impl(const Launch& L, const Tables& T, int64_t n_boxes, int h,
                                       int order, int64_t budget, const float* pre_up,
                                       const float* pre_lo, int64_t ld, const int32_t* nterms,
                                       float* lo, float* hi, EncloseOpts ro) {
  const int64_t n_items = n_boxes * h;   // with a list: its largest possible length
  if (n_items == 0) return cudaSuccess;
  int G;
  const int lb = effective_order(T.n, order, budget, &G, L.ews != nullptr);
  if (lb > T.rscale_max || T.rscale[lb] == nullptr) return cudaErrorInvalidValue;
  // Shared-memory grids of at least 256 cells: a block per polynomial
  // (variants 3 and 4 of the enclosure tuner: 128 or 320 threads; 3 is the
  // default from kEncloseBlkGrid cells) or a warp per polynomial (variants
  // 0-2, items per block)
  const bool blk_ok = G >= 256 && G <= kEncloseGridMax && lb >= 3 && lb <= 16;
  bool blk = false, blk_wide = false;
  TuneTimer tt;
  std::string key;
  if (blk_ok) {
    key = "enclose/" + std::to_string(lb) + "/" + std::to_string(T.n) + "/" +
          std::to_string(n_items);
    const int v = tune_variant(L, "enclose", key, G >= kEncloseBlkGrid ? 3 : 0);
    blk = v >= 3;
    blk_wide = v == 4;
  }
  if (G > kEncloseGridMax || blk) {
    // global-memory grids, or a block per polynomial: lo/hi, then the ReLU
    // step on the same items
    if (blk) tune_begin(L, "enclose", tt);
    cudaError_t e =
        G > kEncloseGridMax
            ? launch_enclose_big(L, T, lb, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi,
                                 ro.list, ro.count)
            : launch_enclose_blk(L, T, lb, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi,
                                 ro.list, ro.count, blk_wide);
    if (e == cudaSuccess && ro.kind != nullptr) {
      k_relu_coeffs_list<<<(unsigned)((n_items + 127) / 128), 128, 0, L.stream>>>(
          ro.list, ro.count, n_items, lo, hi, ro.degrees, ro.global_d, ro.kind, ro.coef, ro.eps,
          L.status);
      ++*L.launches;
      e = cudaGetLastError();
    }
    if (blk) tune_end(L, "enclose", key, tt);
    return e;
  }
  if (G <= kSmallGrid && lb <= 7) {
#define BERN_SMALL_CASE(X) \
  case X: return launch_small<X>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, ro);
    switch (lb) {
      BERN_SMALL_CASE(0) BERN_SMALL_CASE(1) BERN_SMALL_CASE(2) BERN_SMALL_CASE(3)
      BERN_SMALL_CASE(4) BERN_SMALL_CASE(5) BERN_SMALL_CASE(6) BERN_SMALL_CASE(7)
      default: break;
    }
#undef BERN_SMALL_CASE
  }
#define BERN_ENC_CASE(X) \
  case X: return launch_lb<X>(L, T, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, ro);
  switch (lb) {
    BERN_ENC_CASE(0) BERN_ENC_CASE(1) BERN_ENC_CASE(2) BERN_ENC_CASE(3) BERN_ENC_CASE(4)
    BERN_ENC_CASE(5) BERN_ENC_CASE(6) BERN_ENC_CASE(7) BERN_ENC_CASE(8) BERN_ENC_CASE(9)
    BERN_ENC_CASE(10) BERN_ENC_CASE(11) BERN_ENC_CASE(12) BERN_ENC_CASE(13) BERN_ENC_CASE(14)
    BERN_ENC_CASE(15) BERN_ENC_CASE(16)
    default:
      return launch_generic(L, T, lb, G, n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, ro);
  }
#undef BERN_ENC_CASE
}

cudaError_t launch_enclose(const Launch& L, const Tables& T, int64_t n_boxes, int h, int order,
                           int64_t budget, const float* pre_up, const float* pre_lo, int64_t ld,
                           const int32_t* nterms, float* lo, float* hi) {
  return launch_enclose_impl(L, T, n_boxes, h, order, budget, pre_up, pre_lo, ld, nterms, lo,
                             hi, EncloseOpts{nullptr, nullptr, nullptr, nullptr, 0});
}

cudaError_t launch_enclose_relu(const Launch& L, const Tables& T, int64_t n_boxes, int h,
                                int order, int64_t budget, const float* pre_up,
                                const float* pre_lo, int64_t ld, const int32_t* nterms,
                                float* lo, float* hi, const uint8_t* degrees, int global_d,
                                int8_t* kind, float* coef, float* eps) {
  return launch_enclose_impl(L, T, n_boxes, h, order, budget, pre_up, pre_lo, ld, nterms, lo,
                             hi, EncloseOpts{kind, coef, eps, degrees, global_d});
}

// Stability screen of a hidden layer's items before the enclosure.  On the box
// every monomial t^K lies in [0,1], so a polynomial p lies in
//   [c_0 + sum_{K>0} min(0, c_K),  c_0 + sum_{K>0} max(0, c_K)]
// (summed rounding down, resp. up), an interval that contains the range of
// its Bernstein coefficients (each is c_0 plus the other coefficients with
// weights in [0,1]).  An item whose upper polynomial is <= 0 or whose lower
// polynomial is >= 0 on this interval is stable (the cases of Sec. 5.1 Step
// 2): it gets its case, the interval as lo/hi, and no enclosure or ReLU
// coefficients (nothing downstream reads them).  The other items are appended
// to `list` (one atomic per warp) for the enclosure.  One thread per item, so
// a warp reads one coefficient of 32 neighbouring neurons at a time.
__global__ void __launch_bounds__(256)
k_stable_screen(int64_t n_items, int h, const float* __restrict__ pre_up,
                const float* __restrict__ pre_lo, int64_t ld, const int32_t* __restrict__ nterms,
                float* __restrict__ lo, float* __restrict__ hi, int8_t* __restrict__ kind,
                int* __restrict__ list, int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool need = false;
  if (it < n_items) {
    const int nt = nterms[it];
    if (nt < 0 || nt > ld) {
      need = true;                                  // the enclosure reports it
    } else {
      const int64_t b = it / h;
      const int64_t base = (b * ld) * h + (it - b * h);
      float l = 0.0f, u = 0.0f;
      if (nt > 0) {
        l = pre_lo[base];
        u = pre_up[base];
        // eight coefficients of each bound in flight per round; the sums
        // keep the sequential order
        int r = 1;
        for (; r + 8 <= nt; r += 8) {
          float xl[8], xu[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            xl[q] = pre_lo[base + (int64_t)(r + q) * h];
            xu[q] = pre_up[base + (int64_t)(r + q) * h];
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            l = __fadd_rd(l, fminf(xl[q], 0.0f));
            u = __fadd_ru(u, fmaxf(xu[q], 0.0f));
          }
        }
        for (; r < nt; ++r) {
          l = __fadd_rd(l, fminf(pre_lo[base + (int64_t)r * h], 0.0f));
          u = __fadd_ru(u, fmaxf(pre_up[base + (int64_t)r * h], 0.0f));
        }
      }
      if (!(isfinite(l) && isfinite(u)) || (u > 0.0f && l < 0.0f)) {
        need = true;
      } else {
        kind[it] = u <= 0.0f ? 0 : 1;
        lo[it] = l;
        hi[it] = u;
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, need);
  int at = 0;
  if (lane == 0 && m) at = atomicAdd(count, __popc(m));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (need) list[at + __popc(m & ((1u << lane) - 1u))] = (int)it;
}

// The same screen with four neighbouring neurons per thread (h a multiple of
// 4, 16-byte aligned blocks): one float4 load per coefficient row and bound
// serves four items, each summed in the same order as above.
__global__ void __launch_bounds__(256)
k_stable_screen4(int64_t n_items, int h, const float4* __restrict__ pre_up4,
                 const float4* __restrict__ pre_lo4, int64_t ld,
                 const int32_t* __restrict__ nterms, float* __restrict__ lo,
                 float* __restrict__ hi, int8_t* __restrict__ kind, int* __restrict__ list,
                 int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t it0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  bool need[4] = {false, false, false, false};
  if (it0 < n_items) {
    int nt[4], ntmax = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      nt[i] = nterms[it0 + i];
      if (nt[i] < 0 || nt[i] > ld) {
        need[i] = true;                             // the enclosure reports it
        nt[i] = 0;
      }
      ntmax = max(ntmax, nt[i]);
    }
    const int64_t b = it0 / h;
    const int64_t hq = h >> 2;                      // float4s per coefficient row
    const int64_t base = ((b * ld) * h + (it0 - b * h)) >> 2;
    float l[4] = {0.0f, 0.0f, 0.0f, 0.0f}, u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (ntmax > 0) {
      const float4 a = pre_lo4[base], c = pre_up4[base];
      const float al[4] = {a.x, a.y, a.z, a.w}, cu[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        l[i] = nt[i] > 0 ? al[i] : 0.0f;
        u[i] = nt[i] > 0 ? cu[i] : 0.0f;
      }
    }
    int r = 1;
    for (; r + 4 <= ntmax; r += 4) {
      float4 xl[4], xu[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xl[q] = pre_lo4[base + (r + q) * hq];
        xu[q] = pre_up4[base + (r + q) * hq];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float vl[4] = {xl[q].x, xl[q].y, xl[q].z, xl[q].w};
        const float vu[4] = {xu[q].x, xu[q].y, xu[q].z, xu[q].w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (r + q < nt[i]) {
            l[i] = __fadd_rd(l[i], fminf(vl[i], 0.0f));
            u[i] = __fadd_ru(u[i], fmaxf(vu[i], 0.0f));
          }
      }
    }
    for (; r < ntmax; ++r) {
      const float4 x = pre_lo4[base + r * hq], y = pre_up4[base + r * hq];
      const float vl[4] = {x.x, x.y, x.z, x.w}, vu[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r < nt[i]) {
          l[i] = __fadd_rd(l[i], fminf(vl[i], 0.0f));
          u[i] = __fadd_ru(u[i], fmaxf(vu[i], 0.0f));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (need[i]) continue;
      if (!(isfinite(l[i]) && isfinite(u[i])) || (u[i] > 0.0f && l[i] < 0.0f)) {
        need[i] = true;
      } else {
        kind[it0 + i] = u[i] <= 0.0f ? 0 : 1;
        lo[it0 + i] = l[i];
        hi[it0 + i] = u[i];
      }
    }
  }
  // append this thread's undecided items: a warp scan of the counts, one
  // atomic per warp
  const int cnt = (int)need[0] + (int)need[1] + (int)need[2] + (int)need[3];
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int at = 0;
  if (lane == 31 && total) at = atomicAdd(count, total);
  at = __shfl_sync(0xffffffffu, at, 31) + incl - cnt;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (need[i]) list[at++] = (int)(it0 + i);
}

cudaError_t launch_enclose_relu_screened(const Launch& L, const Tables& T,
                                         const ComposeScratch& S, int64_t n_boxes, int h,
                                         int order, int64_t budget, const float* pre_up,
                                         const float* pre_lo, int64_t ld,
                                         const int32_t* nterms, float* lo, float* hi,
                                         const uint8_t* degrees, int global_d, int8_t* kind,
                                         float* coef, float* eps) {
  const int64_t n_items = n_boxes * h;
  if (n_items == 0) return cudaSuccess;
  if (n_items > S.qcap || n_items > 0x7fffffff) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(S.qcount, 0, sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  const bool quads = (h & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(pre_up) | reinterpret_cast<uintptr_t>(pre_lo)) &
                      15) == 0;
  if (quads)
    k_stable_screen4<<<(unsigned)((n_items / 4 + 255) / 256), 256, 0, L.stream>>>(
        n_items, h, reinterpret_cast<const float4*>(pre_up),
        reinterpret_cast<const float4*>(pre_lo), ld, nterms, lo, hi, kind, S.queue, S.qcount);
  else
    k_stable_screen<<<(unsigned)((n_items + 255) / 256), 256, 0, L.stream>>>(
        n_items, h, pre_up, pre_lo, ld, nterms, lo, hi, kind, S.queue, S.qcount);
  ++*L.launches;
  EncloseOpts o{kind, coef, eps, degrees, global_d};
  o.list = S.queue;
  o.count = S.qcount;
  return launch_enclose_impl(L, T, n_boxes, h, order, budget, pre_up, pre_lo, ld, nterms, lo,
                             hi, o);
}

cudaError_t launch_enclose_relu_listed(const Launch& L, const Tables& T,
                                       const ComposeScratch& S, int64_t n_boxes, int h,
                                       int order, int64_t budget, const float* pre_up,
                                       const float* pre_lo, int64_t ld,
                                       const int32_t* nterms, float* lo, float* hi,
                                       const uint8_t* degrees, int global_d, int8_t* kind,
                                       float* coef, float* eps) {
  const int64_t n_items = n_boxes * h;
  if (n_items == 0) return cudaSuccess;
  if (n_items > S.qcap || n_items > 0x7fffffff) return cudaErrorInvalidValue;
  EncloseOpts o{kind, coef, eps, degrees, global_d};
  o.list = S.queue;
  o.count = S.qcount;
  return launch_enclose_impl(L, T, n_boxes, h, order, budget, pre_up, pre_lo, ld, nterms, lo,
                             hi, o);
}

// ------------------------------------------------------------------ per-box orders
struct OrderKeys {
  int8_t key[kMaxTableDegree + 1];   // order value -> list index, -1 if absent
};

// Stable classification of the items by their box's order (same scheme as
// the composition queues: ballot/popc in a warp, a scan over the warps, one
// atomic per list and block).
__global__ void __launch_bounds__(1024)
k_order_queue(int64_t n_items, int h, const int32_t* __restrict__ box_order, OrderKeys K,
              ComposeScratch S, int* status) {
  __shared__ int s_wcnt[32][kOrderQueues];
  __shared__ int s_base[kOrderQueues];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int q = -1;
  if (item < n_items) {
    const int o = box_order[item / h];
    q = (o >= 0 && o <= kMaxTableDegree) ? K.key[o] : -1;
    if (q < 0) atomicOr(status, kStatusInvalid);
  }
  int rank_in_warp = 0;
  for (int qq = 0; qq < kOrderQueues; ++qq) {
    const unsigned m = __ballot_sync(0xffffffffu, q == qq);
    if (q == qq) rank_in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) s_wcnt[warp][qq] = __popc(m);
  }
  __syncthreads();
  if (threadIdx.x < kOrderQueues) {
    const int qq = threadIdx.x;
    int run = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int c = s_wcnt[w][qq];
      s_wcnt[w][qq] = run;
      run += c;
    }
    s_base[qq] = run ? atomicAdd(&S.qcount[qq], run) : 0;
  }
  __syncthreads();
  if (q >= 0) S.queue[(int64_t)q * S.qcap + s_base[q] + s_wcnt[warp][q] + rank_in_warp] = (int)item;
}

cudaError_t launch_enclose_by_order(const Launch& L, const Tables& T, const ComposeScratch& S,
                                    int64_t n_boxes, int h, const int32_t* box_order,
                                    const std::vector<int>& orders, int64_t budget,
                                    const float* pre_up, const float* pre_lo, int64_t ld,
                                    const int32_t* nterms, float* lo, float* hi) {
  const int64_t n_items = n_boxes * h;
  if (n_items == 0) return cudaSuccess;
  if ((int)orders.size() > kOrderQueues || n_items > S.qcap) return cudaErrorInvalidValue;
  OrderKeys K;
  for (auto& k : K.key) k = -1;
  for (size_t i = 0; i < orders.size(); ++i) {
    if (orders[i] < 0 || orders[i] > kMaxTableDegree) return cudaErrorInvalidValue;
    K.key[orders[i]] = (int8_t)i;
  }
  cudaError_t e = cudaMemsetAsync(S.qcount, 0, kOrderQueues * sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  k_order_queue<<<(unsigned)((n_items + 1023) / 1024), 1024, 0, L.stream>>>(n_items, h, box_order,
                                                                          K, S, L.status);
  ++*L.launches;
  for (size_t i = 0; i < orders.size(); ++i) {
    EncloseOpts o{nullptr, nullptr, nullptr, nullptr, 0};
    o.list = S.queue + (int64_t)i * S.qcap;
    o.count = S.qcount + i;
    e = launch_enclose_impl(L, T, n_boxes, h, orders[i], budget, pre_up, pre_lo, ld, nterms, lo,
                            hi, o);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ a3 alone
__global__ void k_relu_coeffs(int64_t n_items, const float* __restrict__ lo,
                              const float* __restrict__ hi, const uint8_t* __restrict__ degrees,
                              int global_d, int8_t* __restrict__ kind, float* __restrict__ coef,
                              float* __restrict__ eps, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const int d = degrees ? (int)degrees[i] : global_d;
  kind[i] = (int8_t)relu_item(lo[i], hi[i], d, coef + i * kCoefStride, eps + i, status);
}

cudaError_t launch_relu_coeffs(const Launch& L, int64_t n_items, const float* lo,
                               const float* hi, const uint8_t* degrees, int global_d,
                               int8_t* kind, float* coef, float* eps) {
  if (n_items == 0) return cudaSuccess;
  k_relu_coeffs<<<(unsigned)((n_items + 127) / 128), 128, 0, L.stream>>>(
      n_items, lo, hi, degrees, global_d, kind, coef, eps, L.status);
  ++*L.launches;
  return cudaGetLastError();
}

}  // namespace bern
