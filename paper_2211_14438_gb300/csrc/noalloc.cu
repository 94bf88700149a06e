// bern_propagate_noalloc: the whole bound propagation without any device
// allocation, for callers that are not allowed to call cudaMalloc.
//
// Who needs it: code that runs where device allocation is forbidden or
// unsafe - inside a host framework that owns all GPU memory through its own
// pool and rejects foreign cudaMalloc calls, in latency-critical service
// loops where an allocation (and the implicit synchronisation cudaFree may
// cause) is not acceptable, or in plugins loaded into a process whose memory
// budget is fixed up front.  bern_propagate needs a bern_ctx, which allocates
// its workspace, monomial tables and status word with cudaMalloc; this entry
// point instead keeps all three in fixed file-scope __device__ arrays that
// exist from the moment the library is loaded until the process exits.
//
// Limits: the per-box workspace of the network must fit kNoAllocScratchBytes
// (32 MiB) and the monomial/pair tables kNoAllocTableBytes (4 MiB); larger
// problems are rejected with BERN_E_UNSUPPORTED before any GPU work.  Boxes
// are processed in chunks that fit the workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "bern_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr size_t kNoAllocTableBytes = (size_t)4 << 20;
constexpr int kNoAllocMaxDevices = 64;

// The fixed device memory.  In host code these names are only host-side
// stand-ins: the kernels get the device addresses from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) unsigned char g_tables[kNoAllocTableBytes];
static __device__ __align__(256) int g_status;

struct DeviceSlot {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_scratch on this device
  unsigned char* tables = nullptr;
  int* status = nullptr;
  int sms = 0;                        // multiprocessors of the device
  int table_n = -1, table_dmax = -1;  // which tables g_tables currently holds
  bern::Tables view{};
  int64_t launches = 0;
};

DeviceSlot g_slots[kNoAllocMaxDevices];
std::mutex g_mutex;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// One-time set-up per device (the device must be current): look up the
// device addresses of the static arrays.
int setup_device(int dev, DeviceSlot** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return BERN_E_UNSUPPORTED;
  DeviceSlot& s = g_slots[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return BERN_E_CUDA;
    s.scratch = (unsigned char*)p;
    if (cudaGetSymbolAddress(&p, g_tables) != cudaSuccess) return BERN_E_CUDA;
    s.tables = (unsigned char*)p;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return BERN_E_CUDA;
    s.status = (int*)p;
    if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return BERN_E_CUDA;
    s.ready = true;
  }
  *out = &s;
  return BERN_OK;
}

// Build the graded exponent table (up to degree `deg_exps`), M(n,D) counts
// and the square pair tables for degrees 0..dmax into one host image, and
// copy it into g_tables on `stream`.
int upload_tables(DeviceSlot& s, int n, int dmax, int deg_exps, cudaStream_t stream) {
  if (s.table_n == n && s.table_dmax >= dmax && s.view.mexps >= bern::num_monomials(n, deg_exps))
    return BERN_OK;
  std::vector<unsigned char> img;
  auto put = [&](const void* src, size_t bytes) {
    size_t off = align256(img.size());
    img.resize(off + bytes);
    if (bytes) std::memcpy(img.data() + off, src, bytes);
    return off;
  };
  std::vector<int32_t> mc(bern::kMaxTableDegree + 1);
  for (int D = 0; D <= bern::kMaxTableDegree; ++D) {
    int64_t m = bern::num_monomials(n, D);
    mc[D] = (m < 0 || m > INT32_MAX) ? INT32_MAX : (int32_t)m;
  }
  size_t off_mc = put(mc.data(), mc.size() * sizeof(int32_t));
  std::vector<uint8_t> ex;
  bern::graded_monomials(n, deg_exps, ex);
  size_t off_ex = put(ex.data(), ex.size());
  std::vector<uint8_t> dof;
  bern::build_degree_of(n, deg_exps, dof);
  size_t off_dof = put(dof.data(), dof.size());
  const int rmax = bern::max_enclose_order(n);
  std::vector<size_t> off_rs(rmax + 1), off_gi(rmax + 1), off_li(rmax + 1);
  for (int l = 0; l <= rmax; ++l) {
    std::vector<float> rs;
    bern::build_rscale(n, l, rs);
    off_rs[l] = put(rs.data(), rs.size() * sizeof(float));
    std::vector<int32_t> gi, li;
    bern::build_enclose_tables(n, l, gi, li);
    off_gi[l] = put(gi.data(), gi.size() * sizeof(int32_t));
    off_li[l] = put(li.data(), li.size() * sizeof(int32_t));
    if (img.size() > kNoAllocTableBytes) return BERN_E_UNSUPPORTED;
  }
  const int row_dmax = std::min(bern::kMaxRowDegree, bern::row_path_max_degree(n));
  struct RowOff { size_t pos_in, hdr, in_off, pairs, out_ranks; int m_in, n_out_rows, row_split; };
  std::vector<RowOff> roff(row_dmax + 1);
  for (int D = 0; D <= row_dmax; ++D) {
    bern::RowImage ri;
    if (!bern::build_row_table(n, D, ri)) return BERN_E_UNSUPPORTED;
    roff[D].m_in = ri.m_in;
    roff[D].n_out_rows = ri.n_out_rows;
    roff[D].row_split = ri.row_split;
    roff[D].pos_in = put(ri.pos_in.data(), ri.pos_in.size() * sizeof(int32_t));
    roff[D].hdr = put(ri.hdr.data(), ri.hdr.size() * sizeof(int32_t));
    roff[D].in_off = put(ri.in_off.data(), ri.in_off.size() * sizeof(int32_t));
    roff[D].pairs = put(ri.pairs.data(), ri.pairs.size() * sizeof(int32_t));
    roff[D].out_ranks = put(ri.out_ranks.data(), ri.out_ranks.size() * sizeof(int32_t));
    if (img.size() > kNoAllocTableBytes) return BERN_E_UNSUPPORTED;
  }
  std::vector<size_t> off_ptr(dmax + 1), off_pairs(dmax + 1);
  for (int D = 0; D <= dmax; ++D) {
    bern::PairList pl;
    if (!bern::build_square_pairs(n, D, pl)) return BERN_E_UNSUPPORTED;
    off_ptr[D] = put(pl.ptr.data(), pl.ptr.size() * sizeof(int32_t));
    off_pairs[D] = put(pl.pairs.data(), pl.pairs.size() * sizeof(uint32_t));
    if (img.size() > kNoAllocTableBytes) return BERN_E_UNSUPPORTED;
  }
  if (img.size() > kNoAllocTableBytes) return BERN_E_UNSUPPORTED;
  // from here g_tables is being overwritten: until the new view is in place
  // the slot holds no valid tables, so a failed copy is never taken for them
  s.table_n = -1;
  s.table_dmax = -1;
  // the copy is ordered on the caller's stream after every earlier call on it
  if (cudaMemcpyAsync(s.tables, img.data(), img.size(), cudaMemcpyHostToDevice, stream) !=
      cudaSuccess)
    return BERN_E_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return BERN_E_CUDA;
  bern::Tables v{};
  v.n = n;
  v.dmax = dmax;
  v.mcount = (const int32_t*)(s.tables + off_mc);
  v.exps = (const uint8_t*)(s.tables + off_ex);
  v.mexps = bern::num_monomials(n, deg_exps);
  v.deg_of = (const uint8_t*)(s.tables + off_dof);
  v.row_dmax = row_dmax;
  for (int D = 0; D <= row_dmax; ++D) {
    bern::RowTable& rt = v.row[D];
    rt.m_in = roff[D].m_in;
    rt.n_out_rows = roff[D].n_out_rows;
    rt.row_split = roff[D].row_split;
    rt.pos_in = (const int32_t*)(s.tables + roff[D].pos_in);
    rt.hdr = (const int4*)(s.tables + roff[D].hdr);
    rt.in_off = (const int32_t*)(s.tables + roff[D].in_off);
    rt.pairs = (const int4*)(s.tables + roff[D].pairs);
    rt.out_ranks = (const int32_t*)(s.tables + roff[D].out_ranks);
  }
  v.rscale_max = rmax;
  for (int l = 0; l <= rmax; ++l) {
    v.rscale[l] = (const float2*)(s.tables + off_rs[l]);
    v.gidx[l] = (const int32_t*)(s.tables + off_gi[l]);
    v.lines[l] = (const int2*)(s.tables + off_li[l]);
  }
  for (int D = 0; D <= dmax; ++D) {
    v.sq[D].ptr = (const int32_t*)(s.tables + off_ptr[D]);
    v.sq[D].pairs = (const uint32_t*)(s.tables + off_pairs[D]);
  }
  s.view = v;
  s.table_n = n;
  s.table_dmax = dmax;
  return BERN_OK;
}

// Bytes of the table image upload_tables would build, from the monomial
// counts alone (every table's length is fixed by n and the degrees), so that
// a plan whose tables cannot fit is rejected before any of them is built.
// Returns SIZE_MAX when a count overflows.
size_t table_image_bytes(int n, int dmax, int deg_exps) {
  size_t total = 0;
  bool bad = false;
  auto add = [&](double bytes) {
    if (!(bytes >= 0.0) || bytes > 1e15) {
      bad = true;
      return;
    }
    total = align256(total) + (size_t)bytes;
  };
  auto M = [&](int nn, int D) -> double {
    const int64_t m = bern::num_monomials(nn, D);
    if (m < 0) bad = true;
    return (double)m;
  };
  add(4.0 * (bern::kMaxTableDegree + 1));                 // M(n, D) counts
  add(M(n, deg_exps) * n);                                // graded exponents
  add(M(n, deg_exps) + 1);                                // degree of a prefix length
  const int rmax = bern::max_enclose_order(n);
  for (int l = 0; l <= rmax; ++l) {
    double lines = 1.0;
    for (int k = 0; k < n - 1; ++k) lines *= (l + 1);
    add(8.0 * M(n, l));                                   // reciprocal brackets
    add(4.0 * M(n, l));                                   // grid index per rank
    add(8.0 * n * lines);                                 // line bases and digit sums
  }
  const int row_dmax = std::min(bern::kMaxRowDegree, bern::row_path_max_degree(n));
  for (int D = 0; D <= row_dmax; ++D) {
    const double np_out = n == 1 ? 1.0 : M(n - 1, 2 * D);
    const double np_in = n == 1 ? 1.0 : M(n - 1, D);
    add(4.0 * M(n, D));                                   // row-layout positions
    add(16.0 * np_out);                                   // row headers
    add(4.0 * np_out);                                    // input-row offsets
    add(16.0 * np_in * (np_in + 1) / 2);                  // row pairs
    add(4.0 * M(n, 2 * D));                               // output ranks
  }
  for (int D = 0; D <= dmax; ++D) {
    const double m = M(n, D);
    add(4.0 * (M(n, 2 * D) + 1));                         // pair pointers
    add(4.0 * m * (m + 1) / 2);                           // square pairs
  }
  return bad ? SIZE_MAX : total;
}

struct NaLayer {
  int h_in, h_out, d, D_pre, D_post, order;
  int64_t M_pre, M_post;
  bool hidden;
  size_t pre_up, pre_lo, pre_nt, lo, hi, kind, coef, eps, post_up, post_lo, post_nt;
};

}  // namespace

extern "C" int bern_propagate_noalloc(const bern_net* net, const float* boxes, int64_t n_boxes,
                                      const bern_degree_plan* plan, bern_result* result,
                                      void* stream_handle) {
  if (!net || !net->widths || !result || net->n_layers < 1 || n_boxes < 0 ||
      (!boxes && n_boxes > 0))
    return BERN_E_INVALID;
  const int H = net->n_layers, n = net->widths[0], o = net->widths[H];
  if (n < 1 || n > bern::kMaxVars) return BERN_E_INVALID;
  for (int i = 0; i <= H; ++i)
    if (net->widths[i] < 1) return BERN_E_INVALID;
  bern_degree_plan def{};
  def.kind = BERN_DEG_GLOBAL;
  def.global_d = 2;
  const bern_degree_plan* dp = plan ? plan : &def;
  if (dp->kind != BERN_DEG_GLOBAL && dp->kind != BERN_DEG_PER_LAYER) return BERN_E_UNSUPPORTED;
  if (dp->kind == BERN_DEG_PER_LAYER && !dp->per_layer) return BERN_E_INVALID;
  const int cap = dp->degree_cap > 0 ? dp->degree_cap : 16;
  if (cap > bern::kMaxTableDegree || !(dp->prune_tau >= 0.0f)) return BERN_E_INVALID;
  // the static tables hold the order-1/2 kernels' tables only: no Horner
  // items (orders >= 3, pruning) on this path
  if (dp->prune_tau > 0.0f || dp->lin_every != 0) return BERN_E_UNSUPPORTED;
  const int64_t budget = dp->bern_budget > 0 ? dp->bern_budget : ((int64_t)1 << 20);
  if (n_boxes == 0) return BERN_OK;
  if (!result->lo || !result->hi || !result->n_terms || result->cap_terms < 0)
    return BERN_E_INVALID;

  // ---- plan: degrees, term counts and the per-box workspace layout
  std::vector<NaLayer> L(H);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align256(off + bytes);
    return r;
  };
  int hmax = 1;
  for (int i = 1; i <= H; ++i) hmax = std::max(hmax, net->widths[i]);
  const size_t q_region = take(sizeof(int) * bern::kComposeQueues * hmax);
  const size_t z_up = take(sizeof(float) * n * (n + 1));
  const size_t z_lo = take(sizeof(float) * n * (n + 1));
  const size_t z_nt = take(sizeof(int32_t) * n);
  int D = 1, order = 1, dsq = 0, dexp = 1;
  for (int i = 0; i < H; ++i) {
    NaLayer& l = L[i];
    l.h_in = net->widths[i];
    l.h_out = net->widths[i + 1];
    l.hidden = i < H - 1;
    l.D_pre = D;
    l.order = order;
    l.d = 1;
    if (l.hidden) {
      l.d = dp->kind == BERN_DEG_GLOBAL ? dp->global_d : dp->per_layer[i];
      if (l.d < 1 || l.d > bern::kMaxOrder) return BERN_E_INVALID;
      if (l.d >= 3) return BERN_E_UNSUPPORTED;
      l.D_post = std::min(D * l.d, cap);
      if (l.d >= 2) dsq = std::max(dsq, l.D_pre);
      D = l.D_post;
      order = std::min(order * l.d, cap);
    } else {
      l.D_post = l.D_pre;
    }
    dexp = std::max(dexp, std::max(l.D_pre, l.D_post));
    l.M_pre = bern::num_monomials(n, l.D_pre);
    l.M_post = bern::num_monomials(n, l.D_post);
    if (l.M_pre < 0 || l.M_post < 0) return BERN_E_UNSUPPORTED;
    l.pre_up = take(sizeof(float) * l.h_out * l.M_pre);
    l.pre_lo = take(sizeof(float) * l.h_out * l.M_pre);
    l.pre_nt = take(sizeof(int32_t) * l.h_out);
    l.lo = take(sizeof(float) * l.h_out);
    l.hi = take(sizeof(float) * l.h_out);
    if (l.hidden) {
      l.kind = take(l.h_out);
      l.coef = take(sizeof(float) * l.h_out * bern::kCoefStride);
      l.eps = take(sizeof(float) * l.h_out);
      l.post_up = take(sizeof(float) * l.h_out * l.M_post);
      l.post_lo = take(sizeof(float) * l.h_out * l.M_post);
      l.post_nt = take(sizeof(int32_t) * l.h_out);
    }
  }
  const size_t per_box = off;
  const size_t counters = 256;   // composition queue counters, ahead of the per-box regions
  if (per_box + counters > kNoAllocScratchBytes) return BERN_E_UNSUPPORTED;   // one box must fit
  // the tables' size follows from the plan: reject before building any of them
  if (table_image_bytes(n, dsq, dexp) > kNoAllocTableBytes) return BERN_E_UNSUPPORTED;
  const int64_t chunk =
      std::min<int64_t>(n_boxes, (int64_t)((kNoAllocScratchBytes - counters) / per_box));

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BERN_E_CUDA;
  cudaStream_t stream = (cudaStream_t)stream_handle;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot* s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc) return rc;
  rc = upload_tables(*s, n, dsq, dexp, stream);
  if (rc) return rc;
  // the status word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(s->status, 0, sizeof(int), stream) != cudaSuccess) return BERN_E_CUDA;
  bern::Launch La{stream, s->status, &s->launches, nullptr, s->sms};
  const bern::Tables& T = s->view;

  for (int64_t b0 = 0; b0 < n_boxes; b0 += chunk) {
    const int64_t B = std::min(chunk, n_boxes - b0);
    auto at = [&](size_t region) { return s->scratch + counters + region * B; };   // structure of arrays
    bern::ComposeScratch CS{(int*)s->scratch, (int*)at(q_region), B * hmax};
    cudaError_t e = bern::launch_init_inputs(La, n, B, boxes + b0 * n * 2, (float*)at(z_up),
                                             (float*)at(z_lo), n + 1, (int32_t*)at(z_nt));
    const float* in_up = (const float*)at(z_up);
    const float* in_lo = (const float*)at(z_lo);
    const int32_t* in_nt = (const int32_t*)at(z_nt);
    int64_t in_stride = n + 1;
    for (int i = 0; i < H && e == cudaSuccess; ++i) {
      const NaLayer& l = L[i];
      float* pu = (float*)at(l.pre_up);
      float* pl = (float*)at(l.pre_lo);
      int32_t* pn = (int32_t*)at(l.pre_nt);
      e = bern::launch_affine(La, B, l.h_out, l.h_in, net->W[i], net->b[i], in_up, in_lo,
                              in_stride, in_nt, pu, pl, l.M_pre, pn);
      if (e != cudaSuccess) break;
      if (!l.hidden) {
        bern_result r = *result;
        r.lo = result->lo + b0 * o;
        r.hi = result->hi + b0 * o;
        r.n_terms = result->n_terms + b0 * o * 2;
        if (r.coef) r.coef = result->coef + b0 * o * 2 * r.cap_terms;
        if (r.keys) r.keys = result->keys + b0 * o * 2 * r.cap_terms;
        e = bern::launch_enclose(La, T, B, l.h_out, l.order, budget, pu, pl, l.M_pre, pn, r.lo,
                                 r.hi);
        if (e == cudaSuccess) e = bern::launch_pack(La, T, B, o, pu, pl, l.M_pre, pn, r);
        break;
      }
      float* lo = (float*)at(l.lo);
      float* hi = (float*)at(l.hi);
      int8_t* kind = (int8_t*)at(l.kind);
      float* coef = (float*)at(l.coef);
      float* eps = (float*)at(l.eps);
      float* qu = (float*)at(l.post_up);
      float* ql = (float*)at(l.post_lo);
      int32_t* qn = (int32_t*)at(l.post_nt);
      e = bern::launch_enclose_relu(La, T, B, l.h_out, l.order, budget, pu, pl, l.M_pre, pn, lo,
                                    hi, nullptr, l.d, kind, coef, eps);
      if (e == cudaSuccess)
        e = bern::launch_compose(La, T, CS, B, l.h_out, cap, dp->prune_tau, kind, coef, eps,
                                 nullptr, l.d, lo, hi, pu, pl, l.M_pre, pn, qu, ql, l.M_post, qn);
      in_up = qu;
      in_lo = ql;
      in_nt = qn;
      in_stride = l.M_post;
    }
    if (e != cudaSuccess) {
      // launches already queued may still use the shared arrays: let them
      // finish before the lock is released
      cudaStreamSynchronize(stream);
      return BERN_E_CUDA;
    }
  }
  int st = 0;
  if (cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess) {
    cudaStreamSynchronize(stream);
    return BERN_E_CUDA;
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) return BERN_E_CUDA;
  if (st & bern::kStatusInvalid) return BERN_E_INVALID;
  if (st & bern::kStatusUnsupported) return BERN_E_UNSUPPORTED;
  if (st & bern::kStatusCapacity) return BERN_E_CAPACITY;
  if (st & bern::kStatusNonFinite) return BERN_E_NONFINITE;
  return BERN_OK;
}
