// C ABI: context, monomial tables, workspace and the layer-by-layer driver
// of the BERN-NN propagation (Sec. 5.3 of arxiv 2211.14438).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <new>
#include <string>
#include <vector>

#include "bern_internal.cuh"
#include "compose_common.cuh"
#include "mlp.cuh"


using namespace bern;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t reserve(size_t want) {
    if (want <= bytes) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
};

struct TableSet {
  int dmax = -1;
  DevBuf exps, mcount;
  std::vector<DevBuf> bufs;
  Tables view{};
  // product tables of the Horner kernel, built on demand; prod_arr is the
  // device array of kProdStride^2 entries the kernels index
  std::map<std::pair<int, int>, std::pair<DevBuf, DevBuf>> prod;
  std::vector<ProdTable> prod_host;
  DevBuf prod_arr;
};

struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};

// box counters of the fused layer launches (one per launch of a chunk, reused
// modulo this count: launches on one stream run in order)
constexpr int kLayerCounters = 64;

int64_t monomials_clamped(int n, int D) {
  int64_t m = num_monomials(n, D);
  return m < 0 ? -1 : m;
}

}  // namespace

struct bern_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int mem_mode = BERN_MEM_DEVICE;
  int64_t horner_smem_limit = 200 * 1024;
  int use_graphs = 1;
  cudaStream_t gstream = nullptr;   // private stream that graphs are captured on
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int* d_status = nullptr;
  int64_t launches = 0;
  std::map<int, TableSet> tables;
  DevBuf ws, stage_in, stage_out, qbuf, mlp_ws, hbuf;
  DevBuf ctr;                       // box counters of the fused layer kernels
  DevBuf ebuf;                      // grids of enclosures above shared memory
  DevBuf btnt;                      // term counts of the Bernstein-basis layer sum
  int fused = 0;                    // fused layer kernels where a plan allows them
  std::vector<GraphEntry> graphs;
  Tuner tuner;
  int autotune = 1;
  std::set<std::string> tuned;     // plan signatures already tuned
  int sms = 0;                      // multiprocessors of the device
  int* counters() { return (int*)ctr.p; }
  Launch launch() { return launch_on(stream); }
  Launch launch_on(cudaStream_t s) {
    return Launch{s, d_status, &launches, &tuner, sms, (float*)ebuf.p,
                  (int64_t)(ebuf.bytes / sizeof(float))};
  }
  // reserve the enclosure workspace for grids of (n, order, budget); graphs
  // captured with an older buffer are dropped when it moves
  cudaError_t reserve_enclose(int n, int order, int64_t budget);
};

cudaError_t bern_ctx::reserve_enclose(int n, int order, int64_t budget) {
  const size_t floats = enclose_big_floats(n, order, budget, std::max(1, sms));
  if (floats * sizeof(float) <= ebuf.bytes) return cudaSuccess;
  for (auto& g : graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  graphs.clear();
  cudaStreamSynchronize(stream);
  if (gstream) cudaStreamSynchronize(gstream);
  return ebuf.reserve(floats * sizeof(float));
}

namespace {

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return BERN_OK;
  if (e == cudaErrorMemoryAllocation) return BERN_E_NOMEM;
  return BERN_E_CUDA;
}

int status_to_code(int s) {
  if (s & kStatusInvalid) return BERN_E_INVALID;
  if (s & kStatusUnsupported) return BERN_E_UNSUPPORTED;
  if (s & kStatusCapacity) return BERN_E_CAPACITY;
  if (s & kStatusNonFinite) return BERN_E_NONFINITE;
  return BERN_OK;
}

// Largest total degree whose graded exponent table stays below 2^22 ranks.
int exps_degree(int n) {
  int D = 0;
  while (D < kMaxTableDegree && num_monomials(n, D + 1) <= ((int64_t)1 << 22)) ++D;
  return D;
}

// Make sure square tables exist for degrees 0..dmax in n variables.
int ensure_tables(bern_ctx* c, int n, int dmax, const Tables** out) {
  TableSet& ts = c->tables[n];
  if (ts.dmax >= dmax) {
    *out = &ts.view;
    return BERN_OK;
  }
  if (dmax > kMaxTableDegree) return BERN_E_UNSUPPORTED;
  // (re)build from scratch; previously captured graphs hold old pointers.
  // Until the rebuild completes the set holds no valid tables (a failed
  // rebuild leaves it empty, and the next call builds again).
  ts.dmax = -1;
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  cudaStreamSynchronize(c->stream);
  for (auto& b : ts.bufs) b.release();
  ts.bufs.clear();
  ts.view = Tables{};
  ts.view.n = n;
  const int De = exps_degree(n);
  std::vector<uint8_t> ex;
  graded_monomials(n, De, ex);
  cudaError_t e = ts.exps.reserve(ex.size());
  if (e != cudaSuccess) return map_cuda(e);
  cudaMemcpy(ts.exps.p, ex.data(), ex.size(), cudaMemcpyHostToDevice);
  std::vector<int32_t> mc(kMaxTableDegree + 1);
  for (int D = 0; D <= kMaxTableDegree; ++D) {
    int64_t m = num_monomials(n, D);
    mc[D] = (m < 0 || m > INT32_MAX) ? INT32_MAX : (int32_t)m;
  }
  e = ts.mcount.reserve(mc.size() * sizeof(int32_t));
  if (e != cudaSuccess) return map_cuda(e);
  cudaMemcpy(ts.mcount.p, mc.data(), mc.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  ts.view.exps = (const uint8_t*)ts.exps.p;
  ts.view.mcount = (const int32_t*)ts.mcount.p;
  ts.view.mexps = num_monomials(n, De);
  {
    std::vector<uint8_t> dof;
    build_degree_of(n, De, dof);
    DevBuf b;
    if ((e = b.reserve(dof.size())) != cudaSuccess) return map_cuda(e);
    cudaMemcpy(b.p, dof.data(), dof.size(), cudaMemcpyHostToDevice);
    ts.view.deg_of = (const uint8_t*)b.p;
    ts.bufs.push_back(b);
  }
  // reciprocal brackets and grid indices up to the largest order of any
  // enclosure; line tables only for the shared-memory kernels' orders
  ts.view.rscale_max = max_enclose_order_big(n);
  const int lines_max = max_enclose_order(n);
  for (int l = 0; l <= ts.view.rscale_max; ++l) {
    std::vector<float> rs;
    build_rscale(n, l, rs);
    DevBuf b;
    if ((e = b.reserve(rs.size() * sizeof(float))) != cudaSuccess) return map_cuda(e);
    cudaMemcpy(b.p, rs.data(), rs.size() * sizeof(float), cudaMemcpyHostToDevice);
    ts.view.rscale[l] = (const float2*)b.p;
    ts.bufs.push_back(b);
    std::vector<int32_t> gi, li;
    build_enclose_tables(n, l, gi, li, l <= lines_max);
    DevBuf bg, bl;
    if ((e = bg.reserve(gi.size() * sizeof(int32_t))) != cudaSuccess) return map_cuda(e);
    if (!li.empty() && (e = bl.reserve(li.size() * sizeof(int32_t))) != cudaSuccess) {
      bg.release();
      return map_cuda(e);
    }
    cudaMemcpy(bg.p, gi.data(), gi.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (!li.empty())
      cudaMemcpy(bl.p, li.data(), li.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    ts.view.gidx[l] = (const int32_t*)bg.p;
    ts.view.lines[l] = (const int2*)bl.p;
    ts.bufs.push_back(bg);
    ts.bufs.push_back(bl);
  }
  ts.view.row_dmax = std::min(kMaxRowDegree, row_path_max_degree(n));
  for (int D = 0; D <= ts.view.row_dmax; ++D) {
    RowImage ri;
    if (!build_row_table(n, D, ri)) return BERN_E_UNSUPPORTED;
    RowTable& rt = ts.view.row[D];
    rt.m_in = ri.m_in;
    rt.n_out_rows = ri.n_out_rows;
    rt.row_split = ri.row_split;
    auto up = [&](const std::vector<int32_t>& v, const void** dst) -> cudaError_t {
      DevBuf b;
      cudaError_t e2 = b.reserve(std::max<size_t>(16, v.size() * sizeof(int32_t)));
      if (e2 != cudaSuccess) return e2;
      if (!v.empty()) cudaMemcpy(b.p, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      *dst = b.p;
      ts.bufs.push_back(b);
      return cudaSuccess;
    };
    if ((e = up(ri.pos_in, (const void**)&rt.pos_in)) != cudaSuccess) return map_cuda(e);
    if ((e = up(ri.hdr, (const void**)&rt.hdr)) != cudaSuccess) return map_cuda(e);
    if ((e = up(ri.in_off, (const void**)&rt.in_off)) != cudaSuccess) return map_cuda(e);
    if ((e = up(ri.pairs, (const void**)&rt.pairs)) != cudaSuccess) return map_cuda(e);
    if ((e = up(ri.out_ranks, (const void**)&rt.out_ranks)) != cudaSuccess) return map_cuda(e);
  }
  for (int D = 0; D <= dmax; ++D) {
    PairList pl;
    if (!build_square_pairs(n, D, pl)) return BERN_E_UNSUPPORTED;
    DevBuf bp, bq;
    if ((e = bp.reserve(pl.ptr.size() * sizeof(int32_t))) != cudaSuccess) return map_cuda(e);
    if ((e = bq.reserve(std::max<size_t>(4, pl.pairs.size() * sizeof(uint32_t)))) != cudaSuccess)
      return map_cuda(e);
    cudaMemcpy(bp.p, pl.ptr.data(), pl.ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (!pl.pairs.empty())
      cudaMemcpy(bq.p, pl.pairs.data(), pl.pairs.size() * sizeof(uint32_t),
                 cudaMemcpyHostToDevice);
    ts.view.sq[D].ptr = (const int32_t*)bp.p;
    ts.view.sq[D].pairs = (const uint32_t*)bq.p;
    ts.bufs.push_back(bp);
    ts.bufs.push_back(bq);
  }
  if (!ts.prod_arr.p) {
    ts.prod_host.assign((size_t)kProdStride * kProdStride, ProdTable{nullptr, nullptr});
    if ((e = ts.prod_arr.reserve(ts.prod_host.size() * sizeof(ProdTable))) != cudaSuccess)
      return map_cuda(e);
    cudaMemcpy(ts.prod_arr.p, ts.prod_host.data(), ts.prod_host.size() * sizeof(ProdTable),
               cudaMemcpyHostToDevice);
  }
  ts.view.prod = (const ProdTable*)ts.prod_arr.p;
  ts.dmax = dmax;
  ts.view.dmax = dmax;
  e = cudaGetLastError();
  if (e != cudaSuccess) return map_cuda(e);
  *out = &ts.view;
  return BERN_OK;
}

// Product tables for Horner items of input degree <= Dmax and order <= dmax
// under degree cap `cap`: (min(cap, k*D), D) for D <= Dmax, k < dmax.
int ensure_prod_tables(bern_ctx* c, int n, int Dmax, int dmax, int cap) {
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  TableSet& ts = c->tables[n];
  // Tables added by this call reach the kernels through the device array
  // prod_arr; it is refreshed on every exit once something was added (also
  // when a later table fails), and if that copy fails the added tables are
  // dropped again, so a table the host lists is always one the kernels see.
  std::vector<std::pair<int, int>> added;
  auto finish = [&](int rc_in) -> int {
    if (added.empty()) return rc_in;
    const cudaError_t e = cudaMemcpy(ts.prod_arr.p, ts.prod_host.data(),
                                     ts.prod_host.size() * sizeof(ProdTable),
                                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess) return rc_in;
    for (const auto& key : added) {
      ts.prod_host[(size_t)key.first * kProdStride + key.second] = ProdTable{nullptr, nullptr};
      auto it = ts.prod.find(key);
      it->second.first.release();
      it->second.second.release();
      ts.prod.erase(it);
    }
    return map_cuda(e);
  };
  for (int D = 0; D <= Dmax; ++D)
    for (int k = 0; k < std::max(1, dmax); ++k) {
      const int Dq = std::min(cap, k * D);
      if (Dq + D > kMaxTableDegree) return finish(BERN_E_UNSUPPORTED);
      const auto key = std::make_pair(Dq, D);
      if (ts.prod.count(key)) continue;
      std::vector<int32_t> ptr, pairs;
      if (!build_product_table(n, Dq, D, (int64_t)1 << 24, ptr, pairs))
        return finish(BERN_E_UNSUPPORTED);
      DevBuf bp, bq;
      cudaError_t e = bp.reserve(ptr.size() * sizeof(int32_t));
      if (e == cudaSuccess) e = bq.reserve(std::max<size_t>(8, pairs.size() * sizeof(int32_t)));
      if (e != cudaSuccess) {
        bp.release();
        bq.release();
        return finish(map_cuda(e));
      }
      cudaMemcpy(bp.p, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (!pairs.empty())
        cudaMemcpy(bq.p, pairs.data(), pairs.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      ts.prod[key] = std::make_pair(bp, bq);
      ts.prod_host[(size_t)Dq * kProdStride + D] = ProdTable{(const int32_t*)bp.p, (const int2*)bq.p};
      added.push_back(key);
    }
  return finish(BERN_OK);
}

// Composition work queues for up to `items` items.
int ensure_queues(bern_ctx* c, int64_t items, ComposeScratch* out, size_t horner_floats = 0) {
  // *out is part of the graph key byte for byte: zero its padding too
  std::memset(out, 0, sizeof *out);
  const size_t bytes = 256 + (size_t)kQueueLists * items * sizeof(int);
  cudaError_t e = c->qbuf.reserve(bytes);
  if (e != cudaSuccess) return map_cuda(e);
  out->qcount = (int*)c->qbuf.p;
  out->queue = (int*)((char*)c->qbuf.p + 256);
  out->qcap = items;
  out->hws = nullptr;
  out->hws_floats = 0;
  out->horner_smem_limit = c->horner_smem_limit;
  out->hws_blocks = kHornerGlobalPerSM * std::max(1, c->sms);
  if (horner_floats) {
    if ((e = c->hbuf.reserve(horner_floats * sizeof(float))) != cudaSuccess) return map_cuda(e);
    out->hws = (float*)c->hbuf.p;
    out->hws_floats = (int64_t)(c->hbuf.bytes / sizeof(float));
  }
  return BERN_OK;
}

// ------------------------------------------------------------ propagate plan
struct LayerPlan {
  int h_in, h_out;
  int d;            // max ReLU order of this layer's neurons (hidden only)
  int D_pre, D_post;
  int64_t M_pre, M_post;
  // row stride of the pre-activation block: M_post for the per-step hidden
  // layers, whose composition writes the post-activation block in place
  // (it is the same block), M_pre otherwise
  int64_t ld_pre = 0;
  int order;        // Bernstein order of this layer's enclosure
  bool hidden;
  // per-box offsets (in bytes) into the workspace
  size_t off_pre_up, off_pre_lo, off_pre_nt, off_lo, off_hi, off_kind, off_coef, off_eps,
      off_post_up, off_post_lo, off_post_nt, off_deg;
  // learned plans: the per-box Bernstein order of this layer's enclosure and
  // every value it can take
  size_t off_order = 0;
  std::vector<int> orders;
  // fused hidden layer: one kernel from this layer's pre-activation block to
  // the next layer's (no post-activation block, lo/hi or coefficients in HBM)
  bool fused = false;
  // Lin layers (Sec. 5.3): the post-activation bounds are replaced by their
  // multilinear fits shifted by the residual's enclosure at order_post
  bool lin = false;
  int order_post = 0, D_lin = 0;
  int64_t M_lin = 0;
  size_t off_lin_up = 0, off_lin_lo = 0, off_lin_nt = 0, off_lin_rlo = 0, off_lin_rhi = 0;
};

struct Plan {
  int n, o, H, cap;
  int lin = 0;      // linearise every lin-th hidden layer (0: never)
  float tau;
  int64_t budget;
  std::vector<LayerPlan> L;
  size_t off_z_up, off_z_lo, off_z_nt;
  size_t per_box;   // bytes per box
  std::vector<uint8_t> neuron_deg;   // PER_NEURON plans (hidden neurons, layer-major)
  bool per_neuron = false;
  // LEARNED plans
  bool learned = false;
  bern_mlp mlp{};
  float min_conf = 0.0f;
  int fallback_d = 2;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int make_plan(const bern_net* net, const bern_degree_plan* dp, Plan& P, bool allow_fused) {
  if (!net || !net->widths || net->n_layers < 1) return BERN_E_INVALID;
  P.H = net->n_layers;
  P.n = net->widths[0];
  P.o = net->widths[P.H];
  if (P.n < 1 || P.n > kMaxVars) return BERN_E_INVALID;
  for (int i = 0; i <= P.H; ++i)
    if (net->widths[i] < 1) return BERN_E_INVALID;
  bern_degree_plan def{};
  def.kind = BERN_DEG_GLOBAL;
  def.global_d = 2;
  if (!dp) dp = &def;
  P.cap = dp->degree_cap > 0 ? dp->degree_cap : 16;
  if (P.cap > kMaxTableDegree) return BERN_E_INVALID;
  P.tau = dp->prune_tau;
  if (!(P.tau >= 0.0f)) return BERN_E_INVALID;
  P.budget = dp->bern_budget > 0 ? dp->bern_budget : ((int64_t)1 << 20);
  P.lin = dp->lin_every;
  if (P.lin < 0) return BERN_E_INVALID;
  if (P.lin > 0 && dp->kind == BERN_DEG_LEARNED) return BERN_E_UNSUPPORTED;
  P.L.resize(P.H);
  int Dprev = 1, order = 1;
  int hidden_base = 0;
  P.per_neuron = dp->kind == BERN_DEG_PER_NEURON;
  P.learned = dp->kind == BERN_DEG_LEARNED;
  if (P.learned) {
    const bern_mlp* m = dp->mlp;
    if (!m || m->n_features != kDegFeatures || m->n_classes != kDegClasses || !m->W1 || !m->b1 ||
        !m->W2 || !m->b2 || !(dp->min_conf >= 0.0f))
      return BERN_E_INVALID;
    P.mlp = *m;
    P.min_conf = dp->min_conf;
    P.fallback_d = dp->global_d > 0 ? dp->global_d : 2;
    if (P.fallback_d > kMaxOrder) return BERN_E_INVALID;
  }
  std::vector<int> reach{1};   // learned plans: the order values a box can have
  for (int i = 0; i < P.H; ++i) {
    LayerPlan& l = P.L[i];
    l.h_in = net->widths[i];
    l.h_out = net->widths[i + 1];
    l.hidden = i < P.H - 1;
    l.D_pre = Dprev;
    l.order = order;
    l.d = 1;
    if (l.hidden) {
      if (dp->kind == BERN_DEG_GLOBAL) {
        l.d = dp->global_d;
      } else if (dp->kind == BERN_DEG_PER_LAYER) {
        if (!dp->per_layer) return BERN_E_INVALID;
        l.d = dp->per_layer[i];
      } else if (dp->kind == BERN_DEG_LEARNED) {
        // proposals are clamped to per_layer[i] when it is given
        l.d = dp->per_layer ? dp->per_layer[i] : std::max(kDegClasses, P.fallback_d);
        if (l.d < 1 || l.d > kMaxOrder) return BERN_E_INVALID;
      } else if (dp->kind == BERN_DEG_PER_NEURON) {
        if (!dp->per_neuron) return BERN_E_INVALID;
        int mx = 0;
        for (int m = 0; m < l.h_out; ++m) {
          int dm = dp->per_neuron[hidden_base + m];
          if (dm < 1 || dm > kMaxOrder) return BERN_E_INVALID;
          mx = std::max(mx, dm);
          P.neuron_deg.push_back((uint8_t)dm);
        }
        l.d = mx;
      } else {
        return BERN_E_INVALID;
      }
      if (l.d < 1 || l.d > kMaxOrder) return BERN_E_INVALID;
      l.D_post = std::min(Dprev * l.d, P.cap);
      hidden_base += l.h_out;
      Dprev = l.D_post;
      order = std::min(order * l.d, P.cap);
      if (P.lin > 0 && (i + 1) % P.lin == 0) {
        // a multilinear polynomial of total degree <= D has degree <= min(n, D)
        l.lin = true;
        l.order_post = order;
        l.D_lin = std::min(P.n, l.D_post);
        l.M_lin = monomials_clamped(P.n, l.D_lin);
        Dprev = l.D_lin;
        order = std::min(P.n, order);
      }
    } else {
      l.D_post = l.D_pre;
    }
    l.M_pre = monomials_clamped(P.n, l.D_pre);
    l.M_post = monomials_clamped(P.n, l.D_post);
    if (l.M_pre < 0 || l.M_post < 0) return BERN_E_UNSUPPORTED;
    if (P.learned) {
      l.orders = reach;
      if (l.hidden) {
        std::vector<int> next;
        for (int o : reach)
          for (int d = 1; d <= l.d; ++d) {
            const int v = std::min(o * d, P.cap);
            if (std::find(next.begin(), next.end(), v) == next.end()) next.push_back(v);
          }
        std::sort(next.begin(), next.end());
        reach = next;
      }
      if ((int)l.orders.size() > kOrderQueues) return BERN_E_UNSUPPORTED;
    }
  }
  // fused layers: plain plans (one order per layer), no pruning; a Lin layer
  // needs its post-activation block, so it runs the per-step kernels
  if (allow_fused && !P.learned && !P.per_neuron && P.tau == 0.0f)
    for (int i = 0; i + 1 < P.H; ++i) {
      LayerPlan& l = P.L[i];
      l.fused = !l.lin && layer_fused_shape(P.n, l.h_out, P.L[i + 1].h_out, l.d, l.D_pre,
                                            l.order, P.budget, P.cap, nullptr);
    }
  // per-box workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const int n = P.n;
  P.off_z_up = take(sizeof(float) * n * (n + 1));
  P.off_z_lo = take(sizeof(float) * n * (n + 1));
  P.off_z_nt = take(sizeof(int32_t) * n);
  for (auto& l : P.L) {
    const bool in_place = l.hidden && !l.fused;
    l.ld_pre = in_place ? std::max(l.M_pre, l.M_post) : l.M_pre;
    l.off_pre_up = take(sizeof(float) * l.h_out * l.ld_pre);
    l.off_pre_lo = take(sizeof(float) * l.h_out * l.ld_pre);
    l.off_pre_nt = take(sizeof(int32_t) * l.h_out);
    if (l.fused) continue;   // everything past the pre-activation block stays on chip
    l.off_lo = take(sizeof(float) * l.h_out);
    l.off_hi = take(sizeof(float) * l.h_out);
    if (l.hidden) {
      l.off_kind = take(l.h_out);
      l.off_coef = take(sizeof(float) * l.h_out * kCoefStride);
      l.off_eps = take(sizeof(float) * l.h_out);
      l.off_post_up = l.off_pre_up;   // composed in place
      l.off_post_lo = l.off_pre_lo;
      l.off_post_nt = take(sizeof(int32_t) * l.h_out);
      l.off_deg = (P.per_neuron || P.learned) ? take(l.h_out) : 0;
      if (l.lin) {
        l.off_lin_up = take(sizeof(float) * l.h_out * l.M_lin);
        l.off_lin_lo = take(sizeof(float) * l.h_out * l.M_lin);
        l.off_lin_nt = take(sizeof(int32_t) * l.h_out);
        l.off_lin_rlo = take(sizeof(float) * l.h_out);
        l.off_lin_rhi = take(sizeof(float) * l.h_out);
      }
    }
    if (P.learned) l.off_order = take(sizeof(int32_t));
  }
  P.per_box = off;
  return BERN_OK;
}

// Workspace regions are laid out "structure of arrays": region k of a chunk
// of B boxes starts at B * offset_k, and box b's slice of it at b * size_k.
struct Chunk {
  char* base;
  int64_t B;
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(base + off * B); }
};

// Launch sequence of one chunk (graph-capturable: no host sync, no alloc).
int run_chunk(bern_ctx* c, cudaStream_t s, const Plan& P, const Tables& T,
              const ComposeScratch& CS, const bern_net* net, const float* boxes, int64_t B,
              const Chunk& ch, float* out_lo, float* out_hi, bern_result res,
              const bern_trace* trace) {
  int64_t n_hidden = 0, hidden_off = 0;
  for (const auto& l : P.L)
    if (l.hidden) n_hidden += l.h_out;
  Launch L = c->launch_on(s);
  const int n = P.n;
  cudaError_t e = launch_init_inputs(L, n, B, boxes, ch.at<float>(P.off_z_up),
                                     ch.at<float>(P.off_z_lo), n + 1,
                                     ch.at<int32_t>(P.off_z_nt));
  if (e != cudaSuccess) return map_cuda(e);
  const float* in_up = ch.at<float>(P.off_z_up);
  const float* in_lo = ch.at<float>(P.off_z_lo);
  const int32_t* in_nt = ch.at<int32_t>(P.off_z_nt);
  int64_t in_stride = n + 1;
  const MlpView mv{P.mlp.n_features, P.mlp.n_classes, (const __nv_bfloat16*)P.mlp.W1, P.mlp.b1,
                   (const __nv_bfloat16*)P.mlp.W2, P.mlp.b2};
  if (P.learned) {
    e = launch_fill_i32(L, ch.at<int32_t>(P.L[0].off_order), B, 1);
    if (e != cudaSuccess) return map_cuda(e);
  }
  bool pre_ready = false;   // this layer's block was written by a fused kernel
  int fused_idx = 0;
  for (int i = 0; i < P.H; ++i) {
    const LayerPlan& l = P.L[i];
    float* pre_up = ch.at<float>(l.off_pre_up);
    float* pre_lo = ch.at<float>(l.off_pre_lo);
    int32_t* pre_nt = ch.at<int32_t>(l.off_pre_nt);
    const int64_t ldp = l.ld_pre;
    // the stability screen of a plain untraced hidden layer (R21) rides on
    // the affine step where its kernel supports it
    const bool screen_here = l.hidden && !l.fused && !P.learned && !trace && !pre_ready;
    bool screened = false;
    if (!pre_ready) {
      ScreenOut so;
      if (screen_here) {
        so = ScreenOut{ch.at<float>(l.off_lo), ch.at<float>(l.off_hi), ch.at<int8_t>(l.off_kind),
                       CS.queue, CS.qcount};
        e = cudaMemsetAsync(CS.qcount, 0, sizeof(int), s);
        if (e != cudaSuccess) return map_cuda(e);
      }
      e = launch_affine(L, B, l.h_out, l.h_in, net->W[i], net->b[i], in_up, in_lo, in_stride,
                        in_nt, pre_up, pre_lo, ldp, pre_nt, screen_here ? &so : nullptr,
                        &screened);
      if (e != cudaSuccess) return map_cuda(e);
    }
    pre_ready = false;
    if (l.fused) {
      const LayerPlan& nl = P.L[i + 1];
      e = launch_layer(L, T, B, l.h_out, l.d, l.order, P.budget, P.cap, pre_up, pre_lo, ldp,
                       pre_nt, nl.h_out, net->W[i + 1], net->b[i + 1],
                       ch.at<float>(nl.off_pre_up), ch.at<float>(nl.off_pre_lo), nl.ld_pre,
                       ch.at<int32_t>(nl.off_pre_nt),
                       c->counters() + (fused_idx++ % kLayerCounters));
      if (e != cudaSuccess) return map_cuda(e);
      pre_ready = true;
      hidden_off += l.h_out;
      continue;
    }
    if (!l.hidden) {
      if (P.learned)
        e = launch_enclose_by_order(L, T, CS, B, l.h_out, ch.at<int32_t>(l.off_order), l.orders,
                                    P.budget, pre_up, pre_lo, ldp, pre_nt, out_lo, out_hi);
      else
        e = launch_enclose(L, T, B, l.h_out, l.order, P.budget, pre_up, pre_lo, ldp, pre_nt,
                           out_lo, out_hi);
      if (e != cudaSuccess) return map_cuda(e);
      e = launch_pack(L, T, B, P.o, pre_up, pre_lo, ldp, pre_nt, res);
      if (e != cudaSuccess) return map_cuda(e);
      break;
    }
    float* lo = ch.at<float>(l.off_lo);
    float* hi = ch.at<float>(l.off_hi);
    const uint8_t* deg = nullptr;
    if (P.per_neuron || P.learned) deg = ch.at<uint8_t>(l.off_deg);
    int8_t* kind = ch.at<int8_t>(l.off_kind);
    float* coef = ch.at<float>(l.off_coef);
    float* eps = ch.at<float>(l.off_eps);
    if (P.learned) {
      // enclosure at each box's order, then the MLP's orders and the a3 step
      int32_t* ord = ch.at<int32_t>(l.off_order);
      e = launch_enclose_by_order(L, T, CS, B, l.h_out, ord, l.orders, P.budget, pre_up, pre_lo,
                                  ldp, pre_nt, lo, hi);
      if (e != cudaSuccess) return map_cuda(e);
      e = launch_learned_degrees(L, mv, B, l.h_out, i + 1, lo, hi, pre_nt, P.min_conf,
                                 P.fallback_d, l.d, P.cap, ord,
                                 ch.at<int32_t>(P.L[i + 1].off_order),
                                 ch.at<uint8_t>(l.off_deg), kind, coef, eps);
    } else if (!trace) {
      // stable items decided by their coefficient signs skip the enclosure
      // (their lo/hi are read by nothing downstream; a trace reports the
      // Bernstein bounds of every item, so traced runs enclose all of them)
      e = screened
              ? launch_enclose_relu_listed(L, T, CS, B, l.h_out, l.order, P.budget, pre_up, pre_lo,
                                           ldp, pre_nt, lo, hi, deg, l.d, kind, coef, eps)
              : launch_enclose_relu_screened(L, T, CS, B, l.h_out, l.order, P.budget, pre_up,
                                             pre_lo, ldp, pre_nt, lo, hi, deg, l.d, kind, coef,
                                             eps);
    } else {
      e = launch_enclose_relu(L, T, B, l.h_out, l.order, P.budget, pre_up, pre_lo, ldp,
                              pre_nt, lo, hi, deg, l.d, kind, coef, eps);
    }
    if (e != cudaSuccess) return map_cuda(e);
    if (trace) {
      e = launch_trace(L, B, l.h_out, n_hidden, hidden_off, lo, hi, pre_nt, deg, l.d, *trace);
      if (e != cudaSuccess) return map_cuda(e);
    }
    hidden_off += l.h_out;
    float* post_up = ch.at<float>(l.off_post_up);
    float* post_lo = ch.at<float>(l.off_post_lo);
    int32_t* post_nt = ch.at<int32_t>(l.off_post_nt);
    // in place: the post-activation block is the pre-activation block
    e = launch_compose(L, T, CS, B, l.h_out, P.cap, P.tau, kind, coef, eps, deg, l.d, lo, hi,
                       pre_up, pre_lo, ldp, pre_nt, post_up, post_lo, ldp, post_nt, l.M_pre);
    if (e != cudaSuccess) return map_cuda(e);
    if (l.lin) {
      float* lin_up = ch.at<float>(l.off_lin_up);
      float* lin_lo = ch.at<float>(l.off_lin_lo);
      int32_t* lin_nt = ch.at<int32_t>(l.off_lin_nt);
      e = launch_linearize(L, T, B, l.h_out, l.order_post, P.budget, post_up, post_lo, ldp,
                           post_nt, lin_up, lin_lo, l.M_lin, lin_nt, ch.at<float>(l.off_lin_rlo),
                           ch.at<float>(l.off_lin_rhi));
      if (e != cudaSuccess) return map_cuda(e);
      in_up = lin_up;
      in_lo = lin_lo;
      in_nt = lin_nt;
      in_stride = l.M_lin;
    } else {
      in_up = post_up;
      in_lo = post_lo;
      in_nt = post_nt;
      in_stride = ldp;
    }
  }
  return BERN_OK;
}

// Fill the per-item degree arrays of a PER_NEURON plan for a chunk.
int fill_degrees(bern_ctx* c, const Plan& P, const Chunk& ch, int64_t B) {
  if (!P.per_neuron) return BERN_OK;
  size_t base = 0;
  std::vector<uint8_t> host;
  for (const auto& l : P.L) {
    if (!l.hidden) break;
    host.resize((size_t)B * l.h_out);
    for (int64_t b = 0; b < B; ++b)
      std::memcpy(&host[(size_t)b * l.h_out], &P.neuron_deg[base], l.h_out);
    // on the context's stream, so the copy is ordered after the previous
    // chunk's (or call's) kernels that read this workspace, whatever kind of
    // stream the caller gave (pageable source: staged before the call returns)
    cudaError_t e = cudaMemcpyAsync(ch.at<uint8_t>(l.off_deg), host.data(), host.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return map_cuda(e);
    base += l.h_out;
  }
  return BERN_OK;
}

std::string graph_key(const Plan& P, const bern_net* net, const float* boxes, int64_t B,
                      const bern_result& r, const void* wsbase) {
  std::string k;
  auto add = [&](const void* p, size_t s) { k.append((const char*)p, s); };
  add(&B, sizeof B);
  add(&boxes, sizeof boxes);
  add(&P.cap, sizeof P.cap);
  add(&P.tau, sizeof P.tau);
  add(&P.budget, sizeof P.budget);
  add(&P.lin, sizeof P.lin);
  add(&P.learned, sizeof P.learned);
  if (P.learned) {
    add(&P.mlp, sizeof P.mlp);
    add(&P.min_conf, sizeof P.min_conf);
    add(&P.fallback_d, sizeof P.fallback_d);
  }
  add(&wsbase, sizeof wsbase);
  for (int i = 0; i <= P.H; ++i) add(&net->widths[i], sizeof(int));
  for (int i = 0; i < P.H; ++i) {
    add(&net->W[i], sizeof(void*));
    add(&net->b[i], sizeof(void*));
    add(&P.L[i].d, sizeof(int));
    add(&P.L[i].fused, sizeof(bool));   // fused and per-step launch sequences differ
  }
  add(P.neuron_deg.data(), P.neuron_deg.size());
  add(&r, sizeof r);
  return k;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

const char* bern_strerror(int s) {
  switch (s) {
    case BERN_OK: return "ok";
    case BERN_E_INVALID: return "invalid argument";
    case BERN_E_CAPACITY: return "output capacity too small";
    case BERN_E_NONFINITE: return "non-finite bound or coefficient";
    case BERN_E_TIMEOUT: return "device wait timed out";
    case BERN_E_CUDA: return "CUDA runtime error";
    case BERN_E_UNSUPPORTED: return "size beyond library limits";
    case BERN_E_NOMEM: return "out of memory";
    default: return "unknown status";
  }
}

int bern_create(bern_ctx** out, int device, void* stream) {
  if (!out) return BERN_E_INVALID;
  *out = nullptr;
  bern_ctx* c = new (std::nothrow) bern_ctx();
  if (!c) return BERN_E_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = c->ctr.reserve(kLayerCounters * sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return map_cuda(e);
  }
  *out = c;
  return BERN_OK;
}

int bern_destroy(bern_ctx* c) {
  if (!c) return BERN_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->gstream) cudaStreamSynchronize(c->gstream);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& kv : c->tables) {
    kv.second.exps.release();
    kv.second.mcount.release();
    for (auto& b : kv.second.bufs) b.release();
    for (auto& p : kv.second.prod) {
      p.second.first.release();
      p.second.second.release();
    }
    kv.second.prod_arr.release();
  }
  c->ws.release();
  c->qbuf.release();
  c->stage_in.release();
  c->stage_out.release();
  c->mlp_ws.release();
  c->hbuf.release();
  c->ctr.release();
  c->ebuf.release();
  c->btnt.release();
  if (c->d_status) cudaFree(c->d_status);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  delete c;
  return BERN_OK;
}

int bern_set_pointer_mode(bern_ctx* c, int mode) {
  if (!c || (mode != BERN_MEM_DEVICE && mode != BERN_MEM_HOST)) return BERN_E_INVALID;
  c->mem_mode = mode;
  return BERN_OK;
}

int bern_set_autotune(bern_ctx* c, int enable) {
  if (!c) return BERN_E_INVALID;
  c->autotune = enable ? 1 : 0;
  return BERN_OK;
}

int bern_force_variant(bern_ctx* c, const char* kind, int variant) {
  if (!c || !kind) return BERN_E_INVALID;
  const std::string k(kind);
  const int nvar = k == "affine" ? 5 : (k == "enclose" ? 5 : 0);
  if (nvar == 0 || variant < -1 || variant >= nvar) return BERN_E_INVALID;
  cudaStreamSynchronize(c->stream);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (variant < 0)
    c->tuner.forced.erase(k);
  else
    c->tuner.forced[k] = variant;
  return BERN_OK;
}

int bern_set_horner_smem_limit(bern_ctx* c, int64_t bytes) {
  if (!c || bytes < 0) return BERN_E_INVALID;
  c->horner_smem_limit = bytes;
  return BERN_OK;
}

int bern_set_graphs(bern_ctx* c, int enable) {
  if (!c) return BERN_E_INVALID;
  c->use_graphs = enable ? 1 : 0;
  return BERN_OK;
}

int bern_bernstein_square(bern_ctx* c, int n, int l, int64_t n_polys, const float* a,
                          float* c_hi, float* c_lo) {
  if (!c || n_polys < 0 || (n_polys > 0 && (!a || !c_hi || !c_lo))) return BERN_E_INVALID;
  if (!bernstein_square_ok(n, l)) return BERN_E_UNSUPPORTED;
  cudaSetDevice(c->device);
  return map_cuda(launch_bernstein_square(c->launch(), n, l, n_polys, a, c_hi, c_lo));
}

int bern_bernstein_elevate(bern_ctx* c, int n, int l, int r, int64_t n_polys,
                           const float* a_hi, const float* a_lo, float* c_hi, float* c_lo) {
  if (!c || n < 1 || n > kMaxVars || l < 0 || r < 0 || n_polys < 0 ||
      (n_polys > 0 && (!a_hi || !a_lo || !c_hi || !c_lo)))
    return BERN_E_INVALID;
  if (bernstein_elevate_smem(n, l, r) > 200 * 1024) return BERN_E_UNSUPPORTED;
  cudaSetDevice(c->device);
  return map_cuda(launch_bernstein_elevate(c->launch(), n, l, r, n_polys, a_hi, a_lo, c_hi, c_lo));
}

int bern_bernstein_affine(bern_ctx* c, int64_t n_boxes, int h_out, int h_in, const float* W,
                          const float* b, int64_t n_coef, const float* in_hi, const float* in_lo,
                          float* out_hi, float* out_lo) {
  if (!c || n_boxes < 0 || h_out < 1 || h_in < 1 || n_coef < 1 || n_coef > INT32_MAX)
    return BERN_E_INVALID;
  if (n_boxes == 0) return BERN_OK;
  if (!W || !b || !in_hi || !in_lo || !out_hi || !out_lo) return BERN_E_INVALID;
  if ((n_coef + 15) / 16 > 65535 || n_boxes > INT32_MAX) return BERN_E_UNSUPPORTED;
  cudaSetDevice(c->device);
  cudaError_t e = c->btnt.reserve((size_t)n_boxes * (h_in + h_out) * sizeof(int32_t));
  if (e != cudaSuccess) return map_cuda(e);
  return map_cuda(launch_bernstein_affine(c->launch(), n_boxes, h_out, h_in, W, b, (int)n_coef,
                                          in_hi, in_lo, out_hi, out_lo, (int32_t*)c->btnt.p));
}

int bern_set_fused(bern_ctx* c, int enable) {
  if (!c) return BERN_E_INVALID;
  c->fused = enable ? 1 : 0;
  return BERN_OK;
}

int bern_layer(bern_ctx* c, int n, int64_t n_boxes, int h, int order, int64_t budget,
               int global_d, int degree_cap, const float* pre_up, const float* pre_lo,
               int64_t pre_ld, const int32_t* pre_nterms, int h_next, const float* W_next,
               const float* b_next, float* next_up, float* next_lo, int64_t next_ld,
               int32_t* next_nterms) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || h < 1 || h_next < 1 || pre_ld < 1 ||
      next_ld < 1 || order < 0 || degree_cap < 1 || degree_cap > kMaxTableDegree ||
      global_d < 1 || global_d > kMaxOrder)
    return BERN_E_INVALID;
  if (n_boxes == 0) return BERN_OK;
  if (!pre_up || !pre_lo || !pre_nterms || !W_next || !b_next || !next_up || !next_lo ||
      !next_nterms || n_boxes > INT32_MAX)
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  int D_pre = 0;
  while (D_pre < kMaxTableDegree && num_monomials(n, D_pre + 1) <= pre_ld) ++D_pre;
  if (budget <= 0) budget = (int64_t)1 << 20;
  if (!layer_fused_shape(n, h, h_next, global_d, D_pre, order, budget, degree_cap, nullptr))
    return BERN_E_UNSUPPORTED;
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  return map_cuda(launch_layer(c->launch(), *T, n_boxes, h, global_d, order, budget, degree_cap,
                               pre_up, pre_lo, pre_ld, pre_nterms, h_next, W_next, b_next,
                               next_up, next_lo, next_ld, next_nterms, c->counters()));
}

int bern_sync(bern_ctx* c) {
  if (!c) return BERN_E_INVALID;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return map_cuda(e);
  int s = 0;
  e = cudaMemcpy(&s, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return map_cuda(e);
  if (s) cudaMemset(c->d_status, 0, sizeof(int));
  return status_to_code(s);
}

int64_t bern_kernel_launches(const bern_ctx* c) { return c ? c->launches : -1; }

int64_t bern_num_monomials(int n, int D) { return num_monomials(n, D); }

int bern_monomials(int n, int D, uint8_t* exps) {
  if (!exps || num_monomials(n, D) < 0) return BERN_E_INVALID;
  if (num_monomials(n, D) > ((int64_t)1 << 26)) return BERN_E_UNSUPPORTED;
  std::vector<uint8_t> ex;
  graded_monomials(n, D, ex);
  std::memcpy(exps, ex.data(), ex.size());
  return BERN_OK;
}

int bern_enclose_lines(int n, int l, int32_t* out, int64_t cap) {
  if (!out || n < 1 || n > kMaxVars || l < 0) return BERN_E_INVALID;
  int64_t cells = 1;
  for (int k = 0; k < n; ++k) {
    cells *= (int64_t)l + 1;
    if (cells > ((int64_t)1 << 22)) return BERN_E_UNSUPPORTED;
  }
  const int64_t need = 2 * (int64_t)n * (cells / (l + 1));
  if (cap < need) return BERN_E_INVALID;
  std::vector<int32_t> gi, li;
  build_enclose_tables(n, l, gi, li, true);
  if ((int64_t)li.size() != need) return BERN_E_INVALID;
  std::memcpy(out, li.data(), li.size() * sizeof(int32_t));
  return BERN_OK;
}

int bern_enclose_scales(int n, int l, float* out, int64_t cap) {
  if (!out || n < 1 || n > kMaxVars || l < 0 || l > kMaxEncloseOrder) return BERN_E_INVALID;
  if (cap < 2 * num_monomials(n, l)) return BERN_E_INVALID;
  std::vector<float> rs;
  build_rscale(n, l, rs);
  std::memcpy(out, rs.data(), rs.size() * sizeof(float));
  return BERN_OK;
}

int bern_compose_rows(int n, int D, int32_t* out, int64_t cap, int64_t* sizes) {
  if (!sizes || n < 1 || n > kMaxVars || D < 0 || D > kMaxRowDegree) return BERN_E_INVALID;
  if (D > row_path_max_degree(n)) return BERN_E_UNSUPPORTED;
  RowImage im;
  if (!build_row_table(n, D, im)) return BERN_E_UNSUPPORTED;
  sizes[0] = im.m_in;
  sizes[1] = im.n_out_rows;
  sizes[2] = im.row_split;
  sizes[3] = (int64_t)im.pairs.size() / 4;
  sizes[4] = (int64_t)im.out_ranks.size();
  if (!out) return BERN_OK;
  const std::vector<int32_t>* parts[] = {&im.pos_in, &im.hdr, &im.in_off, &im.pairs,
                                         &im.out_ranks};
  int64_t need = 0;
  for (const auto* v : parts) need += (int64_t)v->size();
  if (cap < need) return BERN_E_INVALID;
  for (const auto* v : parts) {
    std::memcpy(out, v->data(), v->size() * sizeof(int32_t));
    out += v->size();
  }
  return BERN_OK;
}

int bern_pair_lists(int n, int Dq, int Ds, int square, int32_t* ptr, int64_t cap_ptr,
                    int32_t* pairs, int64_t cap_pairs, int64_t* sizes) {
  if (!sizes || n < 1 || n > kMaxVars || Dq < 0 || Ds < 0 || Dq + Ds > kMaxTableDegree ||
      (square && Dq != Ds))
    return BERN_E_INVALID;
  std::vector<int32_t> p, q;
  if (square) {
    PairList pl;
    if (!build_square_pairs(n, Dq, pl)) return BERN_E_UNSUPPORTED;
    p = pl.ptr;
    q.resize(2 * pl.pairs.size());
    for (size_t k = 0; k < pl.pairs.size(); ++k) {
      q[2 * k] = (int32_t)(pl.pairs[k] & 0xffffu);
      q[2 * k + 1] = (int32_t)(pl.pairs[k] >> 16);
    }
  } else if (!build_product_table(n, Dq, Ds, (int64_t)1 << 24, p, q)) {
    return BERN_E_UNSUPPORTED;
  }
  sizes[0] = (int64_t)p.size();
  sizes[1] = (int64_t)q.size() / 2;
  if (!ptr || !pairs) return BERN_OK;
  if (cap_ptr < (int64_t)p.size() || cap_pairs < (int64_t)q.size()) return BERN_E_INVALID;
  std::memcpy(ptr, p.data(), p.size() * sizeof(int32_t));
  std::memcpy(pairs, q.data(), q.size() * sizeof(int32_t));
  return BERN_OK;
}

int bern_init_inputs(bern_ctx* c, int n, int64_t n_boxes, const float* boxes, float* z_up,
                     float* z_lo, int64_t ld, int32_t* nterms) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || ld < n + 1) return BERN_E_INVALID;
  cudaSetDevice(c->device);
  return map_cuda(launch_init_inputs(c->launch(), n, n_boxes, boxes, z_up, z_lo, ld, nterms));
}

int bern_affine(bern_ctx* c, int64_t n_boxes, int h_out, int h_in, const float* W,
                const float* b, const float* in_up, const float* in_lo, int64_t in_ld,
                const int32_t* in_nterms, float* out_up, float* out_lo, int64_t out_ld,
                int32_t* out_nterms) {
  if (!c || n_boxes < 0 || h_out < 1 || h_in < 1 || in_ld < 1 || out_ld < 1)
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  return map_cuda(launch_affine(c->launch(), n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld,
                                in_nterms, out_up, out_lo, out_ld, out_nterms));
}

int bern_poly_to_x(bern_ctx* c, int n, int64_t n_boxes, int o, const float* boxes,
                   const int32_t* n_terms, const float* coef_t, int64_t cap_terms,
                   float* coef_x) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || o < 1 || cap_terms < 1 || !boxes ||
      !n_terms || !coef_t || !coef_x)
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  // the degree of the longest graded prefix the buffers can hold
  int D = 0;
  while (D < kMaxTableDegree && num_monomials(n, D) < std::min<int64_t>(cap_terms, T->mexps)) ++D;
  if (poly_to_x_smem(n, D) > 200 * 1024) return BERN_E_UNSUPPORTED;
  return map_cuda(launch_poly_to_x(c->launch(), *T, n, n_boxes, o, boxes, n_terms, coef_t,
                                   cap_terms, coef_x, D));
}

int bern_enclose(bern_ctx* c, int n, int64_t n_boxes, int h, int order, int64_t budget,
                 const float* pre_up, const float* pre_lo, int64_t ld, const int32_t* nterms,
                 float* lo, float* hi) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || h < 1 || order < 0 || ld < 1)
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  if (ld > T->mexps) return BERN_E_UNSUPPORTED;
  cudaError_t e = c->reserve_enclose(n, order, budget);
  if (e != cudaSuccess) return map_cuda(e);
  return map_cuda(launch_enclose(c->launch(), *T, n_boxes, h, order, budget, pre_up, pre_lo, ld,
                                 nterms, lo, hi));
}

int bern_linearize(bern_ctx* c, int n, int64_t n_boxes, int h, int order, int64_t budget,
                   float* post_up, float* post_lo, int64_t ld, const int32_t* nterms,
                   float* lin_up, float* lin_lo, int64_t lin_ld, int32_t* lin_nterms,
                   float* res_lo, float* res_hi) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || h < 1 || order < 0 || ld < 1 ||
      lin_ld < num_monomials(n, std::min(n, order)))
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  if (ld > T->mexps) return BERN_E_UNSUPPORTED;
  cudaError_t e = c->reserve_enclose(n, order, budget);
  if (e != cudaSuccess) return map_cuda(e);
  return map_cuda(launch_linearize(c->launch(), *T, n_boxes, h, order, budget, post_up, post_lo,
                                   ld, nterms, lin_up, lin_lo, lin_ld, lin_nterms, res_lo,
                                   res_hi));
}

int bern_relu_coeffs(bern_ctx* c, int64_t n_items, const float* lo, const float* hi,
                     const uint8_t* degrees, int global_d, int8_t* kind, float* coef,
                     float* eps) {
  if (!c || n_items < 0 || (!degrees && (global_d < 1 || global_d > kMaxOrder)))
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  return map_cuda(launch_relu_coeffs(c->launch(), n_items, lo, hi, degrees, global_d, kind, coef,
                                     eps));
}

int bern_compose(bern_ctx* c, int n, int64_t n_boxes, int h, int degree_cap, float prune_tau,
                 const int8_t* kind, const float* coef, const float* eps,
                 const uint8_t* degrees, int global_d, const float* lo, const float* hi,
                 const float* pre_up, const float* pre_lo, int64_t pre_ld,
                 const int32_t* pre_nterms, float* post_up, float* post_lo, int64_t post_ld,
                 int32_t* post_nterms) {
  if (!c || n < 1 || n > kMaxVars || n_boxes < 0 || h < 1 || pre_ld < 1 || post_ld < 1 ||
      degree_cap < 1 || degree_cap > kMaxTableDegree || !(prune_tau >= 0.0f) ||
      global_d < 1 || global_d > kMaxOrder)
    return BERN_E_INVALID;
  // in place is both bounds at one stride; any other aliasing is an error
  const bool aliased = (const float*)post_up == pre_up || (const float*)post_lo == pre_lo;
  if (aliased && !((const float*)post_up == pre_up && (const float*)post_lo == pre_lo &&
                   post_ld == pre_ld))
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  int Dmax = 0;
  while (Dmax < kMaxTableDegree && num_monomials(n, Dmax + 1) <= pre_ld) ++Dmax;
  const Tables* T;
  int rc = ensure_tables(c, n, std::min(Dmax, 32), &T);
  if (rc) return rc;
  size_t horner_floats = 0;
  if (global_d >= 3 || prune_tau > 0.0f) {
    if ((rc = ensure_prod_tables(c, n, Dmax, global_d, degree_cap))) return rc;
    const size_t per_block = horner_smem_floats(*T, Dmax, degree_cap, global_d);
    if (per_block == SIZE_MAX || per_block > ((size_t)64 << 20)) return BERN_E_UNSUPPORTED;
    horner_floats = horner_global_floats(*T, Dmax, degree_cap, global_d, c->horner_smem_limit,
                                         kHornerGlobalPerSM * std::max(1, c->sms));
  }
  ComposeScratch CS;
  if ((rc = ensure_queues(c, std::max<int64_t>(1, n_boxes * h), &CS, horner_floats))) return rc;
  return map_cuda(launch_compose(c->launch(), *T, CS, n_boxes, h, degree_cap, prune_tau, kind,
                                 coef, eps, degrees, global_d, lo, hi, pre_up, pre_lo, pre_ld,
                                 pre_nterms, post_up, post_lo, post_ld, post_nterms));
}

int bern_propagate(bern_ctx* c, const bern_net* net, const float* boxes, int64_t n_boxes,
                   const bern_degree_plan* plan, bern_result* result) {
  return bern_propagate_traced(c, net, boxes, n_boxes, plan, result, nullptr);
}

int bern_propagate_traced(bern_ctx* c, const bern_net* net, const float* boxes,
                          int64_t n_boxes, const bern_degree_plan* plan, bern_result* result,
                          const bern_trace* trace) {
  if (!c || !net || !result || n_boxes < 0 || (!boxes && n_boxes > 0)) return BERN_E_INVALID;
  if (trace && c->mem_mode == BERN_MEM_HOST) return BERN_E_INVALID;
  Plan P;
  int rc = make_plan(net, plan, P, c->fused && !trace);
  if (rc) return rc;
  if (n_boxes == 0) return BERN_OK;
  if (!result->lo || !result->hi || !result->n_terms || result->cap_terms < 0)
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  // order-2 items beyond the row path use the pair-list kernel: its inputs
  // (both bounds) must fit shared memory and its square pair list must stay
  // below 2^26 entries (checked before any table is built)
  const int row_dmax_n = std::min(kMaxRowDegree, row_path_max_degree(P.n));
  for (const auto& l : P.L)
    if (l.hidden && l.d == 2 && P.tau == 0.0f && l.D_pre > row_dmax_n &&
        (2 * (size_t)l.M_pre * sizeof(float) > 200 * 1024 ||
         (double)l.M_pre * (double)(l.M_pre + 1) / 2.0 > (double)(1 << 26)))
      return BERN_E_UNSUPPORTED;
  int dsq = 0;
  for (const auto& l : P.L)
    if (l.hidden && l.d >= 2) dsq = std::max(dsq, l.D_pre);
  const Tables* T;
  rc = ensure_tables(c, P.n, dsq, &T);
  if (rc) return rc;
  for (const auto& l : P.L)
    if (l.M_pre > T->mexps || l.M_post > T->mexps) return BERN_E_UNSUPPORTED;
  // workspace of the enclosures whose grids exceed shared memory
  for (const auto& l : P.L) {
    cudaError_t e0 = c->reserve_enclose(P.n, l.order, P.budget);
    for (int o : l.orders)
      if (e0 == cudaSuccess) e0 = c->reserve_enclose(P.n, o, P.budget);
    if (e0 == cudaSuccess && l.lin) e0 = c->reserve_enclose(P.n, l.order_post, P.budget);
    if (e0 != cudaSuccess) return map_cuda(e0);
  }
  size_t horner_floats = 0;
  for (const auto& l : P.L) {
    if (!l.hidden || (l.d < 3 && P.tau == 0.0f)) continue;
    if ((rc = ensure_prod_tables(c, P.n, l.D_pre, l.d, P.cap))) return rc;
    const size_t per_block = horner_smem_floats(*T, l.D_pre, P.cap, l.d);
    if (per_block == SIZE_MAX || per_block > ((size_t)64 << 20)) return BERN_E_UNSUPPORTED;
    horner_floats = std::max(horner_floats,
                             horner_global_floats(*T, l.D_pre, P.cap, l.d, c->horner_smem_limit,
                                                  kHornerGlobalPerSM * std::max(1, c->sms)));
  }

  const bool host = c->mem_mode == BERN_MEM_HOST;
  cudaError_t e;
  // ---- stage inputs for host mode: boxes, weights, biases
  const float* d_boxes = boxes;
  std::vector<const float*> dW(P.H), db(P.H);
  bern_net dnet = *net;
  bern_result dres = *result;
  if (host) {
    size_t bytes_boxes = sizeof(float) * n_boxes * P.n * 2;
    size_t wb = 0;
    for (int i = 0; i < P.H; ++i) wb += (size_t)net->widths[i + 1] * (net->widths[i] + 1);
    size_t in_bytes = align_up(bytes_boxes) + sizeof(float) * wb + 256 * (2 * P.H + 1);
    if ((e = c->stage_in.reserve(in_bytes)) != cudaSuccess) return map_cuda(e);
    char* p = (char*)c->stage_in.p;
    cudaMemcpyAsync(p, boxes, bytes_boxes, cudaMemcpyHostToDevice, c->stream);
    d_boxes = (const float*)p;
    p += align_up(bytes_boxes);
    for (int i = 0; i < P.H; ++i) {
      size_t nw = (size_t)net->widths[i + 1] * net->widths[i];
      cudaMemcpyAsync(p, net->W[i], nw * sizeof(float), cudaMemcpyHostToDevice, c->stream);
      dW[i] = (const float*)p;
      p += align_up(nw * sizeof(float));
      cudaMemcpyAsync(p, net->b[i], net->widths[i + 1] * sizeof(float), cudaMemcpyHostToDevice,
                      c->stream);
      db[i] = (const float*)p;
      p += align_up(net->widths[i + 1] * sizeof(float));
    }
    dnet.W = dW.data();
    dnet.b = db.data();
    const int64_t no = n_boxes * P.o;
    size_t out_bytes = align_up(no * sizeof(float)) * 2 + align_up(no * 2 * sizeof(int32_t));
    if (result->coef) out_bytes += align_up(no * 2 * result->cap_terms * sizeof(float));
    if (result->keys) out_bytes += align_up(no * 2 * result->cap_terms * sizeof(uint64_t));
    if ((e = c->stage_out.reserve(out_bytes)) != cudaSuccess) return map_cuda(e);
    char* q = (char*)c->stage_out.p;
    dres.lo = (float*)q;
    q += align_up(no * sizeof(float));
    dres.hi = (float*)q;
    q += align_up(no * sizeof(float));
    dres.n_terms = (int32_t*)q;
    q += align_up(no * 2 * sizeof(int32_t));
    if (result->coef) {
      dres.coef = (float*)q;
      q += align_up(no * 2 * result->cap_terms * sizeof(float));
    }
    if (result->keys) dres.keys = (uint64_t*)q;
  }
  // ---- workspace: chunk of boxes that fits the budget
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  size_t limit = std::max<size_t>(c->ws.bytes, std::min<size_t>(free_b / 2, (size_t)24 << 30));
  int64_t chunk = std::max<int64_t>(1, (int64_t)(limit / P.per_box));
  chunk = std::min(chunk, n_boxes);
  if ((e = c->ws.reserve(P.per_box * chunk)) != cudaSuccess) return map_cuda(e);
  int hmax = 1;
  for (const auto& l : P.L) hmax = std::max(hmax, l.h_out);
  ComposeScratch CS;
  if ((rc = ensure_queues(c, chunk * hmax, &CS, horner_floats))) return rc;

  // autotune once per plan shape: probe every variant of every tunable kind
  // on the first chunk (plain launches, timed per launch), keep the fastest
  if (c->autotune) {
    std::string sig;
    {
      auto add = [&](const void* p, size_t sz) { sig.append((const char*)p, sz); };
      const int64_t B0 = std::min(chunk, n_boxes);
      add(&B0, sizeof B0);
      add(&P.cap, sizeof P.cap);
      add(&P.tau, sizeof P.tau);
      add(&P.budget, sizeof P.budget);
      add(&P.lin, sizeof P.lin);
      add(&P.learned, sizeof P.learned);
      for (int i = 0; i <= P.H; ++i) add(&net->widths[i], sizeof(int));
      for (const auto& l : P.L) {
        add(&l.d, sizeof l.d);
        add(&l.fused, sizeof l.fused);
      }
    }
    if (!c->tuned.count(sig)) {
      const int64_t B = std::min(chunk, n_boxes);
      Chunk ch{(char*)c->ws.p, B};
      if ((rc = fill_degrees(c, P, ch, B))) return rc;
      const char* kinds[] = {"affine", "enclose"};
      const int nvar[] = {5, 5};
      for (int k = 0; k < 2; ++k) {
        for (int v = 0; v < nvar[k]; ++v) {
          c->tuner.probe_kind = kinds[k];
          c->tuner.probe_variant = v;
          rc = run_chunk(c, c->stream, P, *T, CS, &dnet, d_boxes, B, ch, dres.lo, dres.hi, dres,
                         nullptr);
          if (rc) {
            c->tuner.probe_kind.clear();
            return rc;
          }
        }
        c->tuner.probe_kind.clear();
        for (auto& kv : c->tuner.probe_ms) {
          int best = -1;
          for (int v = 0; v < (int)kv.second.size(); ++v)
            if (kv.second[v] >= 0.0f && (best < 0 || kv.second[v] < kv.second[best])) best = v;
          if (best >= 0) c->tuner.best[kv.first] = best;
        }
        c->tuner.probe_ms.clear();
      }
      if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return map_cuda(e);
      c->tuned.insert(sig);
    }
  }
  for (int64_t b0 = 0; b0 < n_boxes; b0 += chunk) {
    const int64_t B = std::min(chunk, n_boxes - b0);
    Chunk ch{(char*)c->ws.p, B};
    bern_result r = dres;
    r.lo = dres.lo + b0 * P.o;
    r.hi = dres.hi + b0 * P.o;
    r.n_terms = dres.n_terms + b0 * P.o * 2;
    if (r.coef) r.coef = dres.coef + b0 * P.o * 2 * r.cap_terms;
    if (r.keys) r.keys = dres.keys + b0 * P.o * 2 * r.cap_terms;
    const float* bx = d_boxes + b0 * P.n * 2;
    if ((rc = fill_degrees(c, P, ch, B))) return rc;
    bern_trace tr{};
    const bern_trace* tr_ptr = nullptr;
    if (trace) {
      int64_t nh = 0;
      for (const auto& l : P.L)
        if (l.hidden) nh += l.h_out;
      tr = *trace;
      if (tr.lo) tr.lo += b0 * nh;
      if (tr.hi) tr.hi += b0 * nh;
      if (tr.nterms) tr.nterms += b0 * nh;
      if (tr.degree) tr.degree += b0 * nh;
      tr_ptr = &tr;
    }
    if (c->use_graphs) {
      std::string key = graph_key(P, &dnet, bx, B, r, c->ws.p);
      key.append((const char*)&tr, sizeof tr);
      key.append((const char*)&CS, sizeof CS);
      GraphEntry* g = nullptr;
      for (auto& x : c->graphs)
        if (x.key == key) g = &x;
      if (!g) {
        cudaGraph_t graph;
        const int64_t before = c->launches;
        e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return map_cuda(e);
        rc = run_chunk(c, c->gstream, P, *T, CS, &dnet, bx, B, ch, r.lo, r.hi, r, tr_ptr);
        e = cudaStreamEndCapture(c->gstream, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return map_cuda(e);
        GraphEntry ge;
        ge.key = key;
        ge.kernels = c->launches - before;
        c->launches = before;
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return map_cuda(e);
        if (c->graphs.size() >= 16) {
          cudaGraphExecDestroy(c->graphs.front().exec);
          c->graphs.erase(c->graphs.begin());
        }
        c->graphs.push_back(ge);
        g = &c->graphs.back();
      }
      // fork onto the private stream, replay, join back
      if ((e = cudaEventRecord(c->ev_fork, c->stream)) != cudaSuccess) return map_cuda(e);
      if ((e = cudaStreamWaitEvent(c->gstream, c->ev_fork, 0)) != cudaSuccess) return map_cuda(e);
      if ((e = cudaGraphLaunch(g->exec, c->gstream)) != cudaSuccess) return map_cuda(e);
      if ((e = cudaEventRecord(c->ev_join, c->gstream)) != cudaSuccess) return map_cuda(e);
      if ((e = cudaStreamWaitEvent(c->stream, c->ev_join, 0)) != cudaSuccess) return map_cuda(e);
      c->launches += g->kernels;
    } else {
      rc = run_chunk(c, c->stream, P, *T, CS, &dnet, bx, B, ch, r.lo, r.hi, r, tr_ptr);
      if (rc) return rc;
    }
  }
  if (host) {
    const int64_t no = n_boxes * P.o;
    cudaMemcpyAsync(result->lo, dres.lo, no * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(result->hi, dres.hi, no * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(result->n_terms, dres.n_terms, no * 2 * sizeof(int32_t),
                    cudaMemcpyDeviceToHost, c->stream);
    if (result->coef)
      cudaMemcpyAsync(result->coef, dres.coef, no * 2 * result->cap_terms * sizeof(float),
                      cudaMemcpyDeviceToHost, c->stream);
    if (result->keys)
      cudaMemcpyAsync(result->keys, dres.keys, no * 2 * result->cap_terms * sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, c->stream);
    return bern_sync(c);
  }
  e = cudaGetLastError();
  return map_cuda(e);
}

}  // extern "C"

// ------------------------------------------------------------ learned component
namespace {
bool mlp_shape_ok(int F, int C) {
  return F >= 1 && F <= kMlpMaxF && C >= 2 && C <= kMlpMaxC;
}
bool mlp_ok(const bern_mlp* m) {
  return m && mlp_shape_ok(m->n_features, m->n_classes) && m->W1 && m->b1 && m->W2 && m->b2;
}
MlpView view_of(const bern_mlp* m) {
  return MlpView{m->n_features, m->n_classes, (const __nv_bfloat16*)m->W1, m->b1,
                 (const __nv_bfloat16*)m->W2, m->b2};
}
}  // namespace

extern "C" {

int64_t bern_mlp_num_params(int n_features, int n_classes) {
  if (!mlp_shape_ok(n_features, n_classes)) return -1;
  return mlp_num_params(n_features, n_classes);
}

int bern_degree_features(bern_ctx* c, int64_t n_items, const float* lo, const float* hi,
                         const int32_t* nterms, int layer, float* x) {
  if (!c || n_items < 0 || (n_items > 0 && (!lo || !hi || !x))) return BERN_E_INVALID;
  cudaSetDevice(c->device);
  return map_cuda(launch_degree_features(c->launch(), n_items, lo, hi, nterms, layer, x));
}

int bern_split_features(bern_ctx* c, int n, int64_t n_boxes, const float* boxes,
                        const float* root_box, const bern_result* result, int n_outputs,
                        int output, float* x) {
  if (!c || n < 1 || n > kMaxVars || 2 * n + 2 > kMlpMaxF || n_boxes < 0 || !result ||
      n_outputs < 1 || output < 0 || output >= n_outputs)
    return BERN_E_INVALID;
  if (n_boxes > 0 && (!boxes || !root_box || !x || !result->coef || !result->n_terms ||
                      !result->lo || !result->hi))
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  const Tables* T;
  int rc = ensure_tables(c, n, 0, &T);
  if (rc) return rc;
  return map_cuda(launch_split_features(c->launch(), *T, n_boxes, n_outputs, output, boxes,
                                        root_box, *result, x));
}

int bern_mlp_forward(bern_ctx* c, const bern_mlp* mlp, int64_t n, const float* x,
                     float* logits) {
  if (!c || !mlp_ok(mlp) || n < 0 || (n > 0 && (!x || !logits))) return BERN_E_INVALID;
  cudaSetDevice(c->device);
  return map_cuda(launch_mlp_forward(c->launch(), view_of(mlp), n, x, logits));
}

int bern_mlp_backward(bern_ctx* c, const bern_mlp* mlp, int64_t n, const float* x,
                      const int32_t* labels, const float* w, float* grad, float* loss) {
  if (!c || !mlp_ok(mlp) || n < 1 || !x || !labels || !grad || !loss) return BERN_E_INVALID;
  cudaSetDevice(c->device);
  cudaError_t e = c->mlp_ws.reserve(mlp_backward_scratch(n, mlp->n_features, mlp->n_classes));
  if (e != cudaSuccess) return map_cuda(e);
  return map_cuda(launch_mlp_backward(c->launch(), view_of(mlp), n, x, labels, w, c->mlp_ws.p,
                                      grad, loss));
}

int bern_mlp_adam(bern_ctx* c, int n_features, int n_classes, float* param, float* m, float* v,
                  const float* grad, float lr, float beta1, float beta2, float eps, int t,
                  uint16_t* W1_bf16, uint16_t* W2_bf16) {
  if (!c || !mlp_shape_ok(n_features, n_classes) || !param || !m || !v || !grad || !W1_bf16 ||
      !W2_bf16 || t < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return BERN_E_INVALID;
  cudaSetDevice(c->device);
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  return map_cuda(launch_mlp_adam(c->launch(), n_features, n_classes, param, m, v, grad, lr,
                                  beta1, beta2, eps, c1, c2, (__nv_bfloat16*)W1_bf16,
                                  (__nv_bfloat16*)W2_bf16));
}

}  // extern "C"
