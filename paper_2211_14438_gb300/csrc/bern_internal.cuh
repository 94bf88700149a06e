// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/bern.h"

namespace bern {

constexpr int kMaxVars = BERN_MAX_VARS;
constexpr int kMaxOrder = BERN_MAX_ORDER;
constexpr int kMaxTableDegree = 64;      // largest total degree with a monomial table
constexpr int kMaxEncloseOrder = BERN_MAX_ENCLOSE_ORDER;  // C(24,k) is exact in float32
constexpr int kCoefStride = kMaxOrder + 1;

// Device-side status bits (OR-ed by kernels, read by bern_sync).
constexpr int kStatusCapacity = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusInvalid = 4;
constexpr int kStatusUnsupported = 8;

// ------------------------------------------------------------ host tables
int64_t num_monomials(int n, int D);
// graded order, exps[r*n + k]
void graded_monomials(int n, int D, std::vector<uint8_t>& exps);
uint64_t pack_key(const uint8_t* e, int n);

// Output-stationary pair list for the square of a degree-D polynomial:
// for every output rank K < M(n, 2D), the pairs (I, J), I <= J, with
// I + J = K, packed as I | (J << 16).
struct PairList {
  std::vector<int32_t> ptr;     // M_out + 1
  std::vector<uint32_t> pairs;
  int64_t m_in = 0, m_out = 0;
};
bool build_square_pairs(int n, int D, PairList& out);

// Product table of a degree-Dq polynomial q by a degree-Ds polynomial s, for
// the Horner kernel: for every output rank K < M(n, Dq + Ds), the pairs
// (I, J), I + J = K, stored as two int32 (I then J) from pairs[2*ptr[K]].
bool build_product_table(int n, int Dq, int Ds, int64_t max_pairs, std::vector<int32_t>& ptr,
                         std::vector<int32_t>& pairs);

// Row decomposition for the squaring kernel.  A "row" is the set of
// monomials sharing the exponents of t_1..t_{n-1} (its prefix) and varying
// the exponent c of t_n.  The square of a degree-D polynomial is, per output
// row P, the sum over input-row pairs (p, q), p + q = P, of the 1-D
// convolution of the two rows.
constexpr int kMaxRowDegree = 8;          // input degree handled by row convolution
constexpr int kRowLen = kMaxRowDegree + 1;
// Dense index 0..44 of a pair of row lengths 1 <= l1 <= l2 <= kRowLen (the
// case of the squaring kernel's dispatch; dense cases make a jump table).
__host__ __device__ constexpr int row_pair_case(int l1, int l2) {
  return (l1 - 1) * kRowLen - (l1 - 1) * (l1 - 2) / 2 + (l2 - l1);
}
struct RowImage {
  int m_in = 0, n_out_rows = 0;
  int row_split = 0;               // output rows [0, split) hold about half the work
  std::vector<int32_t> pos_in;     // graded rank -> row-layout position
  std::vector<int32_t> hdr;        // per output row: pair_begin, pair_end, rank_begin,
                                   // Lout | in_len<<8 | has_diag<<16 (diagonal pair last)
  std::vector<int32_t> in_off;     // per output row: its input-row offset or -1
  std::vector<int32_t> pairs;      // per pair: off_p, off_q, (L1<<4)|L2 with L1<=L2, row_pair_case
  std::vector<int32_t> out_ranks;  // graded ranks of the output row elements
};
bool build_row_table(int n, int D, RowImage& out);

// ------------------------------------------------------------ device views
struct RowTable {
  int m_in, n_out_rows, row_split;
  const int32_t* pos_in;
  const int4* hdr;
  const int32_t* in_off;
  const int4* pairs;
  const int32_t* out_ranks;
};

struct PairTable {
  const int32_t* ptr;
  const uint32_t* pairs;
};

struct ProdTable {
  const int32_t* ptr;              // null: not built
  const int2* pairs;
};
constexpr int kProdStride = kMaxTableDegree + 1;   // prod[Dq * kProdStride + Ds]

struct Tables {
  int n;
  int dmax;                        // degrees 0..dmax have square tables
  const uint8_t* exps;             // graded exponents, mexps ranks
  int64_t mexps;
  const uint8_t* deg_of;           // deg_of[c] = smallest D with M(n,D) >= c, c <= mexps
  const int32_t* mcount;           // M(n, D) for D = 0..64
  PairTable sq[kMaxTableDegree + 1];
  // rscale[l][r]: float bracket (lo, hi) of 1 / prod_k C(l, e_k(r)) for the
  // ranks r < M(n, l), for Bernstein orders l = 0..rscale_max
  const float2* rscale[kMaxEncloseOrder + 1];
  int rscale_max;
  // per order l <= rscale_max: grid index of every graded rank < M(n, l),
  // and per (variable k, line) the line's (base offset, prefix digit sum)
  const int32_t* gidx[kMaxEncloseOrder + 1];
  const int2* lines[kMaxEncloseOrder + 1];
  // row tables for squaring, input degrees 0..row_dmax (row_dmax <= 8)
  RowTable row[kMaxRowDegree + 1];
  int row_dmax;
  // product tables of the Horner kernel (device array of kProdStride^2)
  const ProdTable* prod;
};

// Largest Bernstein order whose grid fits the shared-memory limit for n vars.
int max_enclose_order(int n);
// Largest Bernstein order the global-memory enclosure handles for n vars
// (grid <= BERN_MAX_BIG_GRID cells, order <= 16, or the shared-memory limit).
int max_enclose_order_big(int n);
// deg_of[c] for c = 0..M(n,De): the smallest D with M(n,D) >= c.
void build_degree_of(int n, int De, std::vector<uint8_t>& out);
// Host image of the reciprocal brackets for order l: 2*M(n,l) floats.
void build_rscale(int n, int l, std::vector<float>& out);
// Enclosure index tables for order l (grid indices of the graded ranks, and
// the lines' base offsets and prefix digit sums; two int32 per line).
void build_enclose_tables(int n, int l, std::vector<int32_t>& gidx, std::vector<int32_t>& lines,
                          bool with_lines = true);

// ------------------------------------------------------------ launchers
// Autotuning.  Launchers that have several valid variants for a shape ask
// the tuner which one to run (by a key naming the kernel kind and shape).  In
// a probe pass the tuner forces one variant of one kind and times every
// launch of that kind with CUDA events; afterwards each key keeps its fastest
// variant.  Every variant computes the same values in the same order.
struct Tuner {
  std::map<std::string, int> best;                        // key -> variant
  std::string probe_kind;                                 // empty: no probe pass
  int probe_variant = -1;
  std::map<std::string, std::vector<float>> probe_ms;     // key -> ms per variant
  std::map<std::string, int> forced;                      // kind -> variant (tests)
};

struct Launch {
  cudaStream_t stream;
  int* status;                     // device status word
  int64_t* launches;               // host counter
  Tuner* tuner = nullptr;
  int sms = 0;                     // multiprocessors of the device (0: query it)
  // workspace of the global-memory enclosure (grids above shared memory);
  // null: enclosures are limited to shared-memory grids (BERN_MAX_GRID)
  float* ews = nullptr;
  int64_t ews_floats = 0;
};
// Multiprocessor count of the launch's device (L.sms, else the current
// device's attribute); grids of persistent kernels are multiples of it.
int device_sms(const Launch& L);

// Variant of `kind` to run for `key` (dflt when untuned).
int tune_variant(const Launch& L, const char* kind, const std::string& key, int dflt);
// Probe timing around one launch of `kind`: tune_begin records the start event
// when this kind is being probed; tune_end records, waits and adds the time.
struct TuneTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool on = false;
};
void tune_begin(const Launch& L, const char* kind, TuneTimer& t);
void tune_end(const Launch& L, const char* kind, const std::string& key, TuneTimer& t);

// Layer-block layout: coefficient r of neuron m of box b at ((b*ld + r)*h + m);
// term counts at b*h + m.
cudaError_t launch_init_inputs(const Launch& L, int n, int64_t n_boxes, const float* boxes,
                               float* z_up, float* z_lo, int64_t ld, int32_t* nterms);
size_t poly_to_x_smem(int n, int D);
cudaError_t launch_poly_to_x(const Launch& L, const Tables& T, int n, int64_t n_boxes, int o,
                             const float* boxes, const int32_t* nterms, const float* coef_t,
                             int64_t cap, float* coef_x, int D);
// Outputs of the stability screen (R21) when the affine step computes it
// from the coefficients it writes: per item the case and the interval of the
// decided items, and the list of the undecided ones (count zeroed by the
// caller).
struct ScreenOut {
  float* lo = nullptr;
  float* hi = nullptr;
  int8_t* kind = nullptr;
  int* list = nullptr;
  int* count = nullptr;
};
// The affine step (a1).  With `screen`, kernels that can also screen the
// output items do, and *screened says whether this launch did.
cudaError_t launch_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                          const float* W, const float* b, const float* in_up,
                          const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                          float* out_up, float* out_lo, int64_t out_ld,
                          int32_t* out_nterms, const ScreenOut* screen = nullptr,
                          bool* screened = nullptr);
cudaError_t launch_enclose(const Launch& L, const Tables& T, int64_t n_boxes, int h, int order,
                           int64_t budget, const float* pre_up, const float* pre_lo, int64_t ld,
                           const int32_t* nterms, float* lo, float* hi);
cudaError_t launch_enclose_relu(const Launch& L, const Tables& T, int64_t n_boxes, int h,
                                int order, int64_t budget, const float* pre_up,
                                const float* pre_lo, int64_t ld, const int32_t* nterms,
                                float* lo, float* hi, const uint8_t* degrees, int global_d,
                                int8_t* kind, float* coef, float* eps);
struct ComposeScratch;
// The same after a stability screen: items that a coefficient-sign interval
// shows stable get their case (and that interval as lo/hi) without the
// enclosure; the rest go through it as an item list in S's first queue.
cudaError_t launch_enclose_relu_screened(const Launch& L, const Tables& T,
                                         const ComposeScratch& S, int64_t n_boxes, int h,
                                         int order, int64_t budget, const float* pre_up,
                                         const float* pre_lo, int64_t ld,
                                         const int32_t* nterms, float* lo, float* hi,
                                         const uint8_t* degrees, int global_d, int8_t* kind,
                                         float* coef, float* eps);
// The same when the items were screened already (by the affine step): the
// enclosure and ReLU step over the list in the scratch queue.
cudaError_t launch_enclose_relu_listed(const Launch& L, const Tables& T,
                                         const ComposeScratch& S, int64_t n_boxes, int h,
                                         int order, int64_t budget, const float* pre_up,
                                         const float* pre_lo, int64_t ld,
                                         const int32_t* nterms, float* lo, float* hi,
                                         const uint8_t* degrees, int global_d, int8_t* kind,
                                         float* coef, float* eps);
cudaError_t launch_relu_coeffs(const Launch& L, int64_t n_items, const float* lo,
                               const float* hi, const uint8_t* degrees, int global_d,
                               int8_t* kind, float* coef, float* eps);
cudaError_t launch_trace(const Launch& L, int64_t n_boxes, int h, int64_t n_hidden, int64_t off,
                         const float* lo, const float* hi, const int32_t* nt,
                         const uint8_t* deg, int global_d, const bern_trace& tr);
cudaError_t launch_split_features(const Launch& L, const Tables& T, int64_t n_boxes, int o, int j,
                                  const float* boxes, const float* root, const bern_result& res,
                                  float* x);
cudaError_t launch_pack(const Launch& L, const Tables& T, int64_t n_boxes, int o,
                        const float* pre_up, const float* pre_lo, int64_t ld,
                        const int32_t* nterms, bern_result res);

// Work queues of the composition step: kComposeQueues lists of item
// indices, each of capacity qcap, and their counters.
constexpr int kComposeQueues = kMaxRowDegree + 6;
// Lists for the per-box Bernstein orders of learned plans (one per order value).
constexpr int kOrderQueues = 32;
constexpr int kQueueLists = kComposeQueues > kOrderQueues ? kComposeQueues : kOrderQueues;
struct ComposeScratch {
  int* qcount;       // kComposeQueues counters (zeroed by the launcher)
  int* queue;        // kComposeQueues * qcap item indices
  int64_t qcap;
  float* hws = nullptr;      // Horner buffers in global memory (polynomials too
  int64_t hws_floats = 0;    // large for shared memory), hws_blocks slices
  int hws_blocks = 0;        // blocks of the global-workspace Horner launch
  int64_t horner_smem_limit = 200 * 1024;   // bytes of shared memory before hws is used
};
// Blocks of the global-workspace Horner launch: two per multiprocessor.
constexpr int kHornerGlobalPerSM = 2;
// Enclosure with a Bernstein order per box (box_order[b]); `orders` lists
// every value box_order may take (at most kOrderQueues).  Items are sorted
// into one list per order in S, then each order runs on its list.
cudaError_t launch_enclose_by_order(const Launch& L, const Tables& T, const ComposeScratch& S,
                                    int64_t n_boxes, int h, const int32_t* box_order,
                                    const std::vector<int>& orders, int64_t budget,
                                    const float* pre_up, const float* pre_lo, int64_t ld,
                                    const int32_t* nterms, float* lo, float* hi);

// Lin step (Sec. 5.3) on a post-activation block: the least-squares
// multilinear fit of every bound goes to lin (graded prefix of
// M(n, min(n, order)) ranks, stride lin_ld, term counts lin_nt), the rounded
// residual overwrites post, its enclosure at `order` goes to rlo/rhi, and the
// fit's constant is shifted by it outward.
cudaError_t launch_linearize(const Launch& L, const Tables& T, int64_t n_boxes, int h, int order,
                             int64_t budget, float* post_up, float* post_lo, int64_t ld,
                             const int32_t* nterms, float* lin_up, float* lin_lo, int64_t lin_ld,
                             int32_t* lin_nt, float* rlo, float* rhi);

// Fused hidden layer (k_layer.cu): stability screen, Bernstein enclosure,
// ReLU coefficients and composition (orders 1-2) of one hidden layer and the
// affine step of the next layer in one launch per layer, from the layer's
// pre-activation block to the next layer's.  layer_fused_shape tells whether
// a layer qualifies (order 1 or 2, input degree within the row tables,
// effective enclosure order <= kLayerMaxOrder, shared memory) and its layout.
constexpr int kLayerMaxOrder = 8;
constexpr int kLayerSmemMax = 227 * 1024 - 256;
struct LayerShape {
  int lb = 0;            // effective Bernstein order of the enclosure
  int ss = 0, hnp = 0, offW = 0, offU = 0, uni = 0, offN = 0, rem_on = 0;
  size_t smem = 0;       // dynamic shared memory per block
};
bool layer_fused_shape(int n, int h, int hn, int d, int D_pre, int order, int64_t budget, int cap,
                       LayerShape* out);
// counter: one device int, zeroed by the launcher (boxes taken by blocks).
cudaError_t launch_layer(const Launch& L, const Tables& T, int64_t n_boxes, int h, int d,
                         int order, int64_t budget, int cap, const float* pre_up,
                         const float* pre_lo, int64_t pre_ld, const int32_t* pre_nt, int hn,
                         const float* Wn, const float* bn, float* nx_up, float* nx_lo,
                         int64_t nx_ld, int32_t* nx_nt, int* counter);
// Effective Bernstein order of an enclosure: the requested order, lowered
// until its grid fits the budget and the grid limit (BERN_MAX_GRID without
// the global-memory path, BERN_MAX_BIG_GRID and order <= 16 with it).
int effective_order(int n, int order, int64_t budget, int* grid_out, bool big = false);
// Global-memory enclosure (k_enclose_big.cu) for grids above BERN_MAX_GRID:
// workspace floats it needs for (n, order, budget) (0 if the grid fits
// shared memory), and its launcher over an item list (list == null: items
// 0..n_items-1); lo/hi only (the ReLU step runs separately).
constexpr int64_t kEncloseBigBytes = (int64_t)1 << 30;
size_t enclose_big_floats(int n, int order, int64_t budget, int sms);
cudaError_t launch_enclose_big(const Launch& L, const Tables& T, int lb, int G, int64_t n_items,
                               int h, const float* pre_up, const float* pre_lo, int64_t ld,
                               const int32_t* nterms, float* lo, float* hi, const int* list,
                               const int* count);
// Grids of at least kEncloseBlkGrid cells that fit shared memory: one block
// per polynomial (lo/hi only; the ReLU step runs on the items afterwards).
constexpr int kEncloseBlkGrid = 2048;
cudaError_t launch_enclose_blk(const Launch& L, const Tables& T, int lb, int G, int64_t n_items,
                               int h, const float* pre_up, const float* pre_lo, int64_t ld,
                               const int32_t* nterms, float* lo, float* hi, const int* list,
                               const int* count, bool wide);

// The square of dense Bernstein tensors by Prod_Bern (k_bern_tensor.cu):
// a [n_polys][(l+1)^n] -> coefficient intervals [c_lo, c_hi] of the square at
// order 2l, [n_polys][(2l+1)^n].  n <= 4, l <= 8, (max_k C(l,k))^n < 2^24.
bool bernstein_square_ok(int n, int l);
cudaError_t launch_bernstein_square(const Launch& L, int n, int l, int64_t n_polys,
                                    const float* a, float* c_hi, float* c_lo);
// Degree elevation of dense Bernstein tensors (order l -> l + r in every
// variable): shared-memory bytes per block, SIZE_MAX when out of range.
size_t bernstein_elevate_smem(int n, int l, int r);
cudaError_t launch_bernstein_elevate(const Launch& L, int n, int l, int r, int64_t n_polys,
                                     const float* a_hi, const float* a_lo, float* c_hi,
                                     float* c_lo);
// The layer sum in the Bernstein basis on dense tensors of G coefficients in
// the layer-block layout; nt_scratch holds n_boxes * (h_in + h_out) ints.
cudaError_t launch_bernstein_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                                    const float* W, const float* b, int G, const float* in_hi,
                                    const float* in_lo, float* out_hi, float* out_lo,
                                    int32_t* nt_scratch);

// Largest input degree the row-convolution path handles for n variables.
int row_path_max_degree(int n);
// The composition step (a4) over a layer block.  pre_ld / post_ld are the
// blocks' row strides; pre_cap (0: pre_ld) the largest term count an input
// can have, which sizes the kernels.  The post block may be the pre block
// itself (post_up == pre_up, post_lo == pre_lo, post_ld == pre_ld): every
// kernel reads an item's inputs before it writes the item's outputs, and the
// identity items then need no copy.
cudaError_t launch_compose(const Launch& L, const Tables& T, const ComposeScratch& S,
                           int64_t n_boxes, int h, int cap, float tau, const int8_t* kind,
                           const float* coef, const float* eps, const uint8_t* degrees,
                           int global_d, const float* lo, const float* hi, const float* pre_up,
                           const float* pre_lo, int64_t pre_ld, const int32_t* pre_nterms,
                           float* post_up, float* post_lo, int64_t post_ld,
                           int32_t* post_nterms, int64_t pre_cap = 0);

}  // namespace bern
