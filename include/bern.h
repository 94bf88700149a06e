/* bern.h — C ABI of the GB300 BERN-NN bound-propagation library.
 *
 * The library computes, for a ReLU feed-forward network NN and a batch of
 * input boxes I_n(dlo, dhi), polynomials p_lo_j(x) <= NN_j(x) <= p_up_j(x)
 * on each box together with lower/upper bounds of each output
 * (arxiv 2211.14438, Problem 1 in Sec. 2; the method of Sec. 5).
 *
 * Representation.  Every polynomial is kept in the power basis of the
 * normalised box coordinates t_i = (x_i - dlo_i) / w_i in [0,1], where
 * w_i >= dhi_i - dlo_i is the box width rounded up to float32.  A polynomial
 * of total degree <= D is a dense float32 vector over the graded monomial
 * order: all exponent vectors with sum 0, then sum 1, ... up to sum D; within
 * one total degree the exponent vectors are in descending lexicographic
 * order of (e_1, ..., e_n).  So a degree-<=D polynomial is exactly the prefix
 * of length M(n,D) = C(n+D, n) of any longer vector, and its "term count" is
 * that prefix length.  bern_monomials() lists the order.
 *
 * Soundness.  All float32 arithmetic that produces an upper polynomial is
 * rounded towards +inf and all that produces a lower one towards -inf, or
 * is followed by a rigorous a-posteriori term folded into the constant
 * coefficient; since every monomial t^K lies in [0,1] on the box, coefficient
 * bounds are value bounds.
 *
 * Memory.  The caller owns every input and output buffer.  The library owns
 * its scratch memory, monomial tables and CUDA graphs (inside bern_ctx).
 * Unless stated otherwise, pointers are device pointers and calls are
 * asynchronous on the context's stream.  Functions return BERN_OK or an
 * error code; nothing throws across this boundary.
 */
#ifndef BERN_H
#define BERN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define BERN_OK            0
#define BERN_E_INVALID     1  /* bad argument: dlo > dhi, NaN box, n > 8, d not in [1,16], ... */
#define BERN_E_CAPACITY    2  /* an output buffer is too small; n_terms tells what is needed */
#define BERN_E_NONFINITE   3  /* a bound or coefficient became NaN/Inf */
#define BERN_E_TIMEOUT     4  /* a device-side wait ran out of its iteration limit */
#define BERN_E_CUDA        5  /* a CUDA runtime call failed */
#define BERN_E_UNSUPPORTED 6  /* a size beyond the library's limits (e.g. degree table too large) */
#define BERN_E_NOMEM       7  /* device or host allocation failed */

/* pointer modes for bern_set_pointer_mode */
#define BERN_MEM_DEVICE 0     /* boxes, network and results are device pointers (async) */
#define BERN_MEM_HOST   1     /* they are host pointers; the call copies in, runs, copies out, syncs */

/* degree plan kinds */
#define BERN_DEG_GLOBAL     0 /* every hidden neuron uses global_d */
#define BERN_DEG_PER_LAYER  1 /* hidden layer i (1-based) uses per_layer[i-1] */
#define BERN_DEG_PER_NEURON 2 /* hidden neuron k (layer-major order) uses per_neuron[k] */
#define BERN_DEG_LEARNED    3 /* the order of every (box, hidden neuron) is proposed at run
                                 time by the plan's degree MLP (see bern_mlp) */

#define BERN_MAX_VARS   8
#define BERN_MAX_ORDER  16    /* largest ReLU Bernstein order d */
#define BERN_MAX_GRID   24576 /* largest Bernstein grid one enclosure stages in shared memory;
                                 larger grids (up to BERN_MAX_BIG_GRID, orders <= 16) run
                                 in a global-memory workspace of the context */
#define BERN_MAX_BIG_GRID 4194304 /* largest Bernstein grid of any enclosure;
                                 bern_budget is clamped to it (to BERN_MAX_GRID in
                                 bern_propagate_noalloc, which has no workspace) */
#define BERN_MAX_ENCLOSE_ORDER 24 /* Bernstein orders above this are lowered to it */

/* the learned component's MLP */
#define BERN_MLP_HIDDEN       64  /* hidden width */
#define BERN_MLP_MAX_FEATURES 16
#define BERN_MLP_MAX_CLASSES  8
#define BERN_DEGREE_FEATURES  8   /* features of one (box, neuron) for degree proposals */
#define BERN_DEGREE_CLASSES   4   /* class c proposes ReLU order c + 1 */

typedef struct bern_ctx bern_ctx;

/* A feed-forward ReLU network (Sec. 2): n_layers affine layers,
 * widths[0] = n inputs ... widths[n_layers] = o outputs; layer i (0-based)
 * has W[i] row-major of shape widths[i+1] x widths[i] and b[i] of length
 * widths[i+1].  ReLU follows every layer except the last.  widths is always
 * a host array; W[i] and b[i] follow the context's pointer mode. */
typedef struct {
  int n_layers;
  const int* widths;
  const float* const* W;
  const float* const* b;
} bern_net;

/* Which Bernstein order d (the paper's L) each hidden neuron uses, and the
 * limits that keep the polynomial sizes bounded.
 *   degree_cap : total-degree cap; terms above it are dropped into a sound
 *                constant remainder (0 means 16).
 *   prune_tau  : terms with |c| < prune_tau * ||q||_1 are dropped likewise
 *                after each product (0 disables pruning).
 *   bern_budget: largest Bernstein grid (l+1)^n one enclosure may use; above
 *                it the enclosure uses a lower order for the low-degree terms
 *                and coefficient intervals for the rest (0 means 2^20; values
 *                above BERN_MAX_BIG_GRID act as BERN_MAX_BIG_GRID).  Grids
 *                above BERN_MAX_GRID run in a global-memory workspace (up to
 *                1 GiB per context; orders up to 16).
 * per_layer / per_neuron are host arrays. */
/* The learned component (not part of the paper's method): a two-layer MLP
 * with BF16 weights and activations and FP32 accumulation,
 *   a = relu(W1 bf16(x) + b1) rounded to bf16   (BERN_MLP_HIDDEN units)
 *   z = W2 a + b2                               (n_classes logits)
 * Device pointers: W1 bf16 bits [HIDDEN x n_features] row-major, b1 fp32
 * [HIDDEN], W2 bf16 bits [n_classes x HIDDEN], b2 fp32 [n_classes].
 * The flat FP32 parameter vector used by training keeps the same four
 * blocks in this order: W1, b1, W2, b2 (bern_mlp_num_params entries). */
typedef struct {
  int n_features;
  int n_classes;
  const uint16_t* W1;
  const float* b1;
  const uint16_t* W2;
  const float* b2;
} bern_mlp;

typedef struct {
  int kind;
  int global_d;
  const int* per_layer;
  const uint8_t* per_neuron;
  int degree_cap;
  float prune_tau;
  int64_t bern_budget;
  /* BERN_DEG_LEARNED: the degree MLP (n_features = BERN_DEGREE_FEATURES,
   * n_classes = BERN_DEGREE_CLASSES, host struct, device weights) and the
   * fallback.  per_layer, if not NULL, caps the order proposed at hidden
   * layer i (1-based) at per_layer[i-1] (it sizes the workspace and tables;
   * without it every layer is sized for order BERN_DEGREE_CLASSES).  A
   * neuron whose largest class probability is below min_conf
   * (>= 0; above 1 every neuron falls back) uses global_d (the plain
   * method's order, 0 means 2). */
  const bern_mlp* mlp;
  float min_conf;
  /* Lin (Sec. 5.3): if > 0, after the composition of every lin_every-th
   * hidden layer each neuron's bounds are replaced by their least-squares
   * multilinear fit on the box (order [1,...,1]) plus the Bernstein
   * enclosure of the residual at the layer's order (max for the upper bound,
   * min for the lower), so the next layer starts from total degree
   * min(n, D).  0 = never.  Not with BERN_DEG_LEARNED plans
   * (BERN_E_UNSUPPORTED) nor with bern_propagate_noalloc. */
  int lin_every;
} bern_degree_plan;

/* Results, all caller-owned, in the context's pointer mode.
 *   lo, hi   : [n_boxes x o]            output enclosures (Sec. 5.3, last paragraph)
 *   n_terms  : [n_boxes x o x 2]        term count of the upper (0) / lower (1) polynomial
 *   keys     : [n_boxes x o x 2 x cap_terms] exponents packed 8 bits per variable
 *              (t_1 in bits 0..7, t_2 in bits 8..15, ...), may be NULL
 *   coef     : same shape, float32 coefficients in t, may be NULL
 * Polynomial (box b, output j, bound k) starts at ((b*o + j)*2 + k)*cap_terms. */
typedef struct {
  float* lo;
  float* hi;
  int32_t* n_terms;
  uint64_t* keys;
  float* coef;
  int64_t cap_terms;
} bern_result;

/* ------------------------------------------------------------ context */

/* Create a context on `device` issuing work to `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Returns BERN_OK, BERN_E_CUDA. */
int bern_create(bern_ctx** ctx, int device, void* stream);

/* Free every library-owned allocation and graph.  Safe on NULL. */
int bern_destroy(bern_ctx* ctx);

/* Select BERN_MEM_DEVICE (default) or BERN_MEM_HOST for bern_propagate. */
int bern_set_pointer_mode(bern_ctx* ctx, int mode);

/* Autotuning (on by default): the first bern_propagate of each plan shape
 * (network widths, plan, batch size) times every variant of the tunable
 * kernels (the wide-layer affine kernel: persistent register-blocked with
 * 4-, 2- or 1-row thread tiles, or 64x32 block tiles; the Bernstein
 * enclosure: 8, 4 or 2 items per block) on its first
 * chunk and keeps the fastest per shape.  All variants compute identical
 * results.  enable = 0 uses the built-in defaults. */
int bern_set_autotune(bern_ctx* ctx, int enable);

/* Force one variant of a tunable kernel family for every later launch on
 * this context (a setting for tests and tuning; the paper has no
 * counterpart).  kind: "affine" (variants 0-4: persistent register-blocked
 * 8x4 thread tiles, block tiles, persistent register-blocked 8x2 and 8x1
 * thread tiles, a warp per box for polynomials of at most 16 terms; 0, 2 and
 * 3 fall back to 1 where the layer's weights do not fit shared memory, 4 to
 * 2 for longer polynomials) or "enclose"
 * (variants 0-2: 8, 4 or 2 items per block with a warp per polynomial; 3, 4:
 * a block of 128 or 320 threads per polynomial for shared-memory grids of
 * 256 cells or more at orders 3-16, else as 2).  variant = -1 clears the
 * force.
 * Drops captured graphs.  Returns BERN_E_INVALID for an unknown kind or a
 * variant out of range. */
int bern_force_variant(bern_ctx* ctx, const char* kind, int variant);

/* Largest shared-memory footprint (bytes, at most 200 KB) the Horner
 * composition kernel may use per block before it keeps its buffers in a
 * global workspace instead; the default is 200 KB.  Both placements compute
 * the same values in the same order (a setting for tests and tuning). */
int bern_set_horner_smem_limit(bern_ctx* ctx, int64_t bytes);

/* Use CUDA-graph replay for bern_propagate (default 1).  With graphs on, the
 * launch sequence of one (network shape, batch size, plan, buffers) tuple is
 * captured once and replayed. */
int bern_set_graphs(bern_ctx* ctx, int enable);

/* Human-readable text of a status code (static storage). */
const char* bern_strerror(int status);

/* Wait for the context's stream and return the first device-side error
 * recorded since the last call (BERN_OK if none); clears it. */
int bern_sync(bern_ctx* ctx);

/* Number of kernels this context has launched so far (graph replays count
 * every kernel node of the graph). */
int64_t bern_kernel_launches(const bern_ctx* ctx);

/* Measured FP32 fused multiply-add throughput of `device` in TFLOP/s (two
 * flops per FMA), the denominator of the kernels' arithmetic rooflines.  The
 * paper has no counterpart: it is the measured peak of the CUDA-core FMA
 * pipe that the bound kernels use.  Every resident thread runs eight
 * independent FMA chains; directed != 0 measures round-up FMAs (as the bound
 * kernels issue), 0 round-to-nearest.  The fastest of `reps` launches (after
 * one warm-up) on `stream` (a cudaStream_t, NULL = legacy default stream);
 * synchronises the stream.  Returns BERN_OK, BERN_E_INVALID (reps < 1 or
 * tflops NULL) or BERN_E_CUDA. */
int bern_fma_throughput(int device, void* stream, int directed, int reps, double* tflops);

/* ------------------------------------------------------------ tables */

/* M(n, D) = C(n+D, n), the number of monomials of total degree <= D in n
 * variables, or -1 if n or D is out of range (n in [1,8], D in [0,64]). */
int64_t bern_num_monomials(int n, int D);

/* Host array exps[M(n,D) x n] of the graded order described above. */
int bern_monomials(int n, int D, uint8_t* exps);

/* The enclosure's line table for order l (Sec. 5.1 Step 1 with Def. 2: the
 * Bernstein coefficients on the grid {0..l}^n follow from one triangular
 * transform per variable along every grid line of that variable), as the
 * shared-memory enclosure kernels use it.  Cell (d_0 .. d_{n-1}) has grid
 * index sum_k d_k (l+1)^(n-1-k).  For each variable k, (l+1)^(n-1) lines of
 * two int32 each: the grid index of the line's first cell (d_k = 0) and the
 * digit sum of the variables before k; pass k starts at out[2 k (l+1)^(n-1)].
 * Within a pass the lines are in the order of the other variables' digits
 * read as one number whose lowest digit is the highest variable; from n = 4
 * on, the C(l+k, k) (l+1)^(n-1-k) lines of prefix sum <= l come first and
 * the rest after them, each part in that order.  (The three-variable kernels
 * compute these entries from the line index instead of loading them.)
 *   out: host array of at least cap int32 (2 n (l+1)^(n-1) are written).
 * Host only; no GPU needed.  Returns BERN_OK; BERN_E_INVALID (out NULL, n
 * outside [1, 8], l < 0, or cap too small); BERN_E_UNSUPPORTED for grids
 * above 2^22 cells. */
int bern_enclose_lines(int n, int l, int32_t* out, int64_t cap);

/* The enclosure's reciprocal brackets for order l (Def. 2: the coefficient a_J
 * enters the Bernstein grid divided by prod_k C(l, j_k)): for each monomial J
 * of degree <= l in the graded order, two floats lo <= 1 / prod_k C(l, j_k)
 * <= hi (equal when the product is a power of two, else the two floats
 * next to the nearest one), which the kernels multiply with the rounding
 * direction of the bound.
 *   out: host array of at least cap floats (2 M(n, l) are written).
 * Host only; no GPU needed.  Returns BERN_OK; BERN_E_INVALID (out NULL, n
 * outside [1, 8], l outside [0, BERN_MAX_ENCLOSE_ORDER], or cap too small). */
int bern_enclose_scales(int n, int l, float* out, int64_t cap);

/* The composition's row tables for input degree D (Sec. 5.1 Step 3 at ReLU
 * order 2: s^2 is formed as sums of 1-D convolutions of the rows of s, a row
 * being the monomials that share the exponents of t_1..t_{n-1}, laid out with
 * the last exponent running), as the row-convolution kernel reads them.
 *   sizes[5] receives m_in = M(n, D), the output rows, the row where the
 *   second half of the work starts, the pairs and the output ranks.
 *   out (NULL: sizes only) receives, concatenated, int32:
 *     pos_in[m_in]     row-layout position of each graded input rank;
 *     hdr[4 per row]   first pair, end of its pairs, first output rank,
 *                      Lout | in_len << 8 | has_diag << 16 (row length of
 *                      the square, of the row's own input row, and whether
 *                      its last pair is a row with itself);
 *     in_off[per row]  row-layout offset of the row's own input row, or -1;
 *     pairs[4 per pair] offsets of the shorter and the longer row,
 *                      L1 << 4 | L2 (L1 <= L2), the dispatch case;
 *     out_ranks[...]   graded rank (degree <= 2D) of each output row element.
 * Host only; no GPU needed.  Returns BERN_OK; BERN_E_INVALID (sizes NULL, n
 * outside [1, 8], D outside [0, 8], or cap too small); BERN_E_UNSUPPORTED
 * when the input has more than 750 terms (those use the pair-list kernel). */
int bern_compose_rows(int n, int D, int32_t* out, int64_t cap, int64_t* sizes);

/* The output-stationary pair lists of the other composition kernels (Sec.
 * 5.1 Step 3; the products of Sec. 4.2 over the graded monomial set): for
 * every output monomial K of degree <= Dq + Ds, the pairs (I, J) of a
 * degree-Dq and a degree-Ds monomial with I + J = K, pairs[2 ptr[K] ..
 * 2 ptr[K+1]) as (I, J) int32 in graded ranks.
 *   square = 1 (Dq == Ds): the square's symmetric list, I <= J (the pair-list
 *     kernel of order-2 items; it packs each pair as I | J << 16);
 *   square = 0: the product table of the Horner kernels (orders >= 3).
 *   sizes[2] receives M(n, Dq + Ds) + 1 and the number of pairs; ptr or pairs
 *   NULL: sizes only.
 * Host only; no GPU needed.  Returns BERN_OK; BERN_E_INVALID (sizes NULL, n
 * outside [1, 8], a degree out of range, square with Dq != Ds, or a cap too
 * small); BERN_E_UNSUPPORTED beyond the kernels' table limits (square: more
 * than 65,535 input terms; product: more than 2^24 pairs). */
int bern_pair_lists(int n, int Dq, int Ds, int square, int32_t* ptr, int64_t cap_ptr,
                    int32_t* pairs, int64_t cap_pairs, int64_t* sizes);

/* ------------------------------------------------------------ hot path */

/* Whole path, Sec. 5.3: input init, then per layer the affine step
 * (Sec. 5.2) and, for hidden layers, Step 1-3 of Sec. 5.1; the last layer is
 * affine only and its enclosure gives lo/hi.
 *   boxes: [n_boxes x n x 2] float32, (dlo_i, dhi_i) per variable.
 * Returns BERN_OK, BERN_E_INVALID, BERN_E_CAPACITY (result->n_terms holds
 * the needed counts), BERN_E_UNSUPPORTED, BERN_E_NONFINITE, BERN_E_CUDA.  In
 * BERN_MEM_DEVICE mode the call is asynchronous and device-side errors are
 * reported by the next bern_sync(); in BERN_MEM_HOST mode it synchronises and
 * reports them itself. */
int bern_propagate(bern_ctx* ctx, const bern_net* net, const float* boxes,
                   int64_t n_boxes, const bern_degree_plan* plan,
                   bern_result* result);

/* Per hidden neuron trace of a propagation (device pointers, caller-owned,
 * [n_boxes x N_hidden], hidden neurons layer-major within a box): the
 * pre-activation enclosure lo/hi (Step 1 of Sec. 5.1), the pre-activation
 * term count, and the ReLU order the neuron used (plan or proposal).  Any
 * pointer may be NULL.  Used to build training data for the learned
 * component and to inspect learned plans. */
typedef struct {
  float* lo;
  float* hi;
  int32_t* nterms;
  uint8_t* degree;
} bern_trace;

/* bern_propagate plus the trace (device pointer mode only). */
int bern_propagate_traced(bern_ctx* ctx, const bern_net* net, const float* boxes,
                          int64_t n_boxes, const bern_degree_plan* plan,
                          bern_result* result, const bern_trace* trace);

/* Output polynomials in the input coordinates x (the change of variables of
 * Sec. 5.3 undone: bern_propagate returns them in t in [0,1]^n with
 * x_i = dlo_i + w_i t_i, w_i = dhi_i - dlo_i rounded up).  For every box b,
 * output j and bound k (0 upper, 1 lower) the polynomial
 *   coef_t[((b*o + j)*2 + k)*cap_terms + r], r < n_terms[(b*o + j)*2 + k]
 * (graded monomial order, bern_result's layout) is rewritten as a polynomial
 * in x over the same graded monomials, into coef_x (same layout; entries past
 * the term count are not written).  The float64 expansion's rounding and the
 * rounding to float are bounded on the box and folded into the constant term
 * (added for upper polynomials, subtracted for lower ones), so the converted
 * upper (lower) polynomial is >= (<=) the original everywhere on the box.
 *   boxes: [n_boxes x n x 2] (dlo, dhi), the boxes the polynomials were
 *   computed on.  All pointers are device pointers; the call is asynchronous
 *   on the context's stream and a term count outside [0, cap_terms], an
 *   invalid box or a non-finite constant is reported by the next bern_sync.
 * Returns BERN_E_INVALID for bad sizes, BERN_E_UNSUPPORTED when cap_terms
 * needs per-variable tables above 200 KB of shared memory (total degree above
 * about 40 for n = 2). */
int bern_poly_to_x(bern_ctx* ctx, int n, int64_t n_boxes, int o, const float* boxes,
                   const int32_t* n_terms, const float* coef_t, int64_t cap_terms,
                   float* coef_x);

/* -------------------------------------------------- step entry points
 * The five steps of the path on the library's dense layout, for testing and
 * for callers composing their own pipeline.  All pointers are device
 * pointers; calls are asynchronous on the context's stream.
 *
 * Layout of a layer block (h neurons per box, leading dimension ld >= the
 * largest term count): the coefficient of monomial r (graded rank) of the
 * polynomial of neuron m of box b is at ((b*ld + r)*h + m) floats, i.e. the
 * coefficients of one monomial of all neurons of a box are contiguous.
 * nterms[b*h + m] coefficients (a graded prefix) are valid for that neuron;
 * entries beyond it are not read.  "up" and "lo" blocks share the layout. */

/* a0, Sec. 5.3 (input init): z0_i = x_i = dlo_i + w_i t_i for both bounds,
 * i.e. a layer block with h = n neurons, ld >= n+1, nterms = n+1. */
int bern_init_inputs(bern_ctx* ctx, int n, int64_t n_boxes, const float* boxes,
                     float* z_up, float* z_lo, int64_t ld, int32_t* nterms);

/* a1, Sec. 5.2, eqs. upper_bounds_layer / lower_bounds_layer:
 *   pre_up_m = sum_j W+_mj up_j + W-_mj lo_j + b_m   (rounded up)
 *   pre_lo_m = sum_j W+_mj lo_j + W-_mj up_j + b_m   (rounded down)
 * W: [h_out x h_in] row-major, b: [h_out]; input block with h = h_in, output
 * block with h = h_out.  Output term count per box is
 * max(1, max_j in_nterms[b*h_in + j]) for all its neurons. */
int bern_affine(bern_ctx* ctx, int64_t n_boxes, int h_out, int h_in,
                const float* W, const float* b, const float* in_up,
                const float* in_lo, int64_t in_ld, const int32_t* in_nterms,
                float* out_up, float* out_lo, int64_t out_ld,
                int32_t* out_nterms);

/* a2, Sec. 5.1 Step 1 (eq. find_lo_hi) with Def. 2: for every neuron of a
 * layer block, lo = min of the Bernstein coefficients of pre_lo, hi = max of
 * those of pre_up, of order `order` in every variable on [0,1]^n (rounded
 * outward).  budget as in bern_degree_plan (0 = 2^20).  lo/hi: [n_boxes x h]. */
int bern_enclose(bern_ctx* ctx, int n, int64_t n_boxes, int h, int order,
                 int64_t budget, const float* pre_up, const float* pre_lo,
                 int64_t ld, const int32_t* nterms, float* lo, float* hi);

/* Lin step, Sec. 5.3 (parameter Lin): for every neuron of a post-activation
 * block, the least-squares multilinear fit A of each bound on [0,1]^n is
 * written to lin_up / lin_lo (a layer block with stride lin_ld >=
 * M(n, min(n, order)); term counts lin_nterms = min(nterms, that)), the
 * residual post - A (rounded up for the upper bound, down for the lower)
 * OVERWRITES post_up / post_lo, its Bernstein enclosure of order `order`
 * goes to res_lo (min over the lower residual) and res_hi (max over the
 * upper one), and A's constant is shifted by it outward: lin_up >= post_up
 * and lin_lo <= post_lo on the box.  budget as in bern_enclose.  res_lo /
 * res_hi: [n_boxes x h]. */
int bern_linearize(bern_ctx* ctx, int n, int64_t n_boxes, int h, int order,
                   int64_t budget, float* post_up, float* post_lo, int64_t ld,
                   const int32_t* nterms, float* lin_up, float* lin_lo,
                   int64_t lin_ld, int32_t* lin_nterms, float* res_lo,
                   float* res_hi);

/* a3, Sec. 5.1 Step 2 with Def. 1 and Props. 1-2: per item the case
 * (0: hi <= 0, output 0; 1: lo >= 0, identity; 2: ReLU polynomial), and for
 * case 2 the power form a_0..a_d in s = (y-lo)/(hi-lo) of the order-d
 * Bernstein polynomial of ReLU on [lo,hi], each rounded up, and the shift
 * eps >= B(0) + sum_j (a_j rounded - a_j), rounded up.
 *   degrees: [n_items] uint8 orders, or NULL to use global_d.
 *   coef: [n_items x (BERN_MAX_ORDER+1)], eps: [n_items], kind: [n_items]. */
int bern_relu_coeffs(bern_ctx* ctx, int64_t n_items, const float* lo,
                     const float* hi, const uint8_t* degrees, int global_d,
                     int8_t* kind, float* coef, float* eps);

/* a4, Sec. 5.1 Step 3, eqs. post_bounds_1/2: post_up = B(s_up), post_lo =
 * B(s_lo) - eps with s = (pre - lo)/(hi - lo), computed as polynomials in t
 * with outward rounding, truncated at total degree `degree_cap` (dropped terms
 * enter the constant as a one-sided remainder).  Identity items copy pre to
 * post; zero items get nterms = 0.  Items are the n_boxes*h neurons of the
 * pre block; kind/coef/eps/degrees/lo/hi are per item (b*h + m).  post_ld
 * must hold M(n, min(d * D_pre, degree_cap)) for every item.
 *   global_d: the order of every item when degrees is NULL; otherwise an
 *     upper bound of the entries of degrees (an entry above it sets
 *     BERN_E_INVALID at bern_sync).
 *   prune_tau >= 0: with prune_tau > 0, after every Horner product the terms
 *     of positive degree with |c| < prune_tau * ||q||_1 are dropped into the
 *     remainder as well, and post_nterms becomes the graded prefix up to the
 *     highest degree with a kept term.
 * Orders 1 and 2 use closed forms (c = a0 + a1 s, a0 + a1 s + a2 s^2); orders
 * >= 3, and every order when prune_tau > 0, use Horner's rule with interval
 * coefficients.  Shapes whose Horner buffers exceed shared memory return
 * BERN_E_UNSUPPORTED.
 * In place: post_up == pre_up, post_lo == pre_lo and post_ld == pre_ld
 * (which must then hold the outputs) compose the block where it stands; every
 * kernel reads an item's inputs before writing its outputs, and identity
 * items keep their coefficients without a copy (bern_propagate composes its
 * hidden layers this way); the kernels are then sized for inputs of up to
 * pre_ld terms.  Other overlaps of pre and post are not allowed (a post
 * pointer equal to a pre pointer otherwise returns BERN_E_INVALID). */
int bern_compose(bern_ctx* ctx, int n, int64_t n_boxes, int h, int degree_cap,
                 float prune_tau, const int8_t* kind, const float* coef,
                 const float* eps, const uint8_t* degrees, int global_d,
                 const float* lo, const float* hi, const float* pre_up,
                 const float* pre_lo, int64_t pre_ld,
                 const int32_t* pre_nterms, float* post_up, float* post_lo,
                 int64_t post_ld, int32_t* post_nterms);

/* a2 + a3 + a4 of one hidden layer and a1 of the next, fused: from the
 * hidden layer's pre-activation block to the next layer's pre-activation
 * block in one launch (Sec. 5.1 Steps 1-3 per neuron, then the layer step of
 * Sec. 5.2 with the next layer's weights), for ReLU orders 1 and 2.  Per box:
 * the stability screen (the coefficient-sign interval of every polynomial,
 * as bern_propagate applies before the enclosure), the Bernstein enclosure of
 * the undecided neurons at `order` under `budget` (0 = 2^20), the ReLU case
 * and coefficients, the composition and the next layer's midpoint-radius
 * affine step, with the rounding of bern_enclose / bern_relu_coeffs /
 * bern_compose / bern_affine; the post-activation polynomials stay in shared
 * memory.
 *   pre_up, pre_lo, pre_nterms: the hidden layer's block (h neurons,
 *     leading dimension pre_ld, layout of bern_affine's output);
 *   W_next [h_next x h] row-major, b_next [h_next]: the next layer;
 *   next_up, next_lo [n_boxes x next_ld x h_next], next_nterms
 *     [n_boxes x h_next]: the next layer's pre-activation block, every
 *     neuron's term count the box's largest post-activation count (as
 *     bern_affine sets it); next_ld must hold the output degree
 *     min(global_d * D, degree_cap) (BERN_E_CAPACITY at bern_sync otherwise).
 * Device pointers; asynchronous on the context's stream.  Shapes the fused
 * kernel does not cover (global_d > 2, h > 256, an input degree beyond the
 * row tables, an effective enclosure order above 8, or shared memory) return
 * BERN_E_UNSUPPORTED before any launch; bern_propagate then uses the
 * per-step kernels for that layer. */
int bern_layer(bern_ctx* ctx, int n, int64_t n_boxes, int h, int order, int64_t budget,
               int global_d, int degree_cap, const float* pre_up, const float* pre_lo,
               int64_t pre_ld, const int32_t* pre_nterms, int h_next, const float* W_next,
               const float* b_next, float* next_up, float* next_lo, int64_t next_ld,
               int32_t* next_nterms);

/* The paper's own representation, for comparison with the power basis: the
 * square of polynomials held as dense Bernstein tensors of order l in every
 * variable (Sec. 4.1), by Prod_Bern (Sec. 4.2: scale by the binomial
 * tensors, multiply as power series, unscale):
 *   c_K = [sum_{I+J=K} (a_I C_l(I)) (a_J C_l(J))] / C_2l(K),
 *   C_l(I) = prod_k C(l, i_k).
 *   a    : [n_polys x (l+1)^n] tensors, index sum_k i_k (l+1)^(n-1-k)
 *          (t_1 the slowest), device pointer;
 *   c_hi, c_lo : [n_polys x (2l+1)^n], the same indexing at order 2l: an
 *          interval containing every exact coefficient of the square
 *          (round-to-nearest sums widened by their a-posteriori error bound).
 * n <= 4 and l <= 8 with (max_k C(l,k))^n < 2^24 (BERN_E_UNSUPPORTED
 * otherwise).  Asynchronous on the context's stream; a non-finite
 * coefficient is reported by bern_sync. */
int bern_bernstein_square(bern_ctx* ctx, int n, int l, int64_t n_polys, const float* a,
                          float* c_hi, float* c_lo);

/* Degree elevation of dense Bernstein tensors (Sec. 4.3, the step Sum_Bern
 * takes before adding tensors of different orders): an order-l tensor in n
 * variables becomes the order-(l + r) tensor of the same polynomial,
 *   c'_k = sum_j c_j C(l, j) C(r, k - j) / C(l + r, k)   in every variable.
 *   a_hi, a_lo: device, n_polys x (l+1)^n floats each, contiguous per
 *          polynomial, row-major with the last variable fastest: an interval
 *          tensor (a_lo <= a_hi; pass one array twice for a point tensor);
 *   c_hi, c_lo: device, n_polys x (l+r+1)^n floats: every exact elevated
 *          coefficient of any tensor in [a_lo, a_hi] lies in [c_lo, c_hi]
 *          (the weights are positive, so the passes round up the upper and
 *          down the lower tensor).
 * l + r <= 24 (exact float binomials) and 4 (l+r+1)^n floats within 200 KB of
 * shared memory (BERN_E_UNSUPPORTED otherwise).  Asynchronous on the context's
 * stream; a non-finite coefficient is reported by bern_sync. */
int bern_bernstein_elevate(bern_ctx* ctx, int n, int l, int r, int64_t n_polys,
                           const float* a_hi, const float* a_lo, float* c_hi, float* c_lo);

/* The layer step of Sec. 5.2 (the sum over a layer's neurons) on dense
 * Bernstein tensors, the Sum_Bern of Sec. 4.3 with weights: for every box and
 * output neuron m,
 *   out_hi_m = b_m + sum_j W+_mj in_hi_j + W-_mj in_lo_j   (out_lo symmetric)
 * coefficient by coefficient, the bias added to every coefficient (the
 * Bernstein basis sums to one).  The tensors share one order and coefficient
 * count n_coef, in the layer-block layout of bern_affine (coefficient g of
 * neuron j of box b at (b * n_coef + g) * h + j).  Every output coefficient
 * bounds the exact one from the correct side (the affine step's directed
 * arithmetic; the Bernstein basis is >= 0 on the box, so the tensors bound
 * the polynomials).  W: h_out x h_in row-major, b: h_out, device.  Holds
 * n_boxes * (h_in + h_out) ints of context scratch.  Asynchronous. */
int bern_bernstein_affine(bern_ctx* ctx, int64_t n_boxes, int h_out, int h_in, const float* W,
                          const float* b, int64_t n_coef, const float* in_hi, const float* in_lo,
                          float* out_hi, float* out_lo);

/* Use the fused layer kernel (bern_layer) inside bern_propagate wherever a
 * plan allows it (default 0): plain plans (BERN_DEG_GLOBAL or PER_LAYER) with
 * prune_tau = 0, untraced, layer by layer where the shape qualifies and the
 * layer is not linearised (lin_every).  enable = 0 runs the per-step kernels for every layer.  Both
 * give the same bounds up to the rounding of sums taken in another order. */
int bern_set_fused(bern_ctx* ctx, int enable);

/* -------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point.  It serves callers that
 * may not allocate device memory: a host framework that owns every GPU
 * allocation through its own pool, a latency-critical loop where cudaMalloc
 * or cudaFree (and the synchronisation they can imply) is not allowed, or a
 * plugin with a fixed memory budget.  It computes exactly what
 * bern_propagate computes, but needs no bern_ctx: its workspace (32 MiB),
 * monomial tables (4 MiB) and status word are fixed __device__ arrays of the
 * library, present on every GPU that loads the library until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *   net, boxes, result: device pointers (layouts as for bern_propagate);
 *   stream: a cudaStream_t (NULL = legacy default stream).
 *   plan: BERN_DEG_GLOBAL or BERN_DEG_PER_LAYER (PER_NEURON, prune_tau > 0
 *   and lin_every != 0 return BERN_E_UNSUPPORTED); NULL means global order
 *   2, cap 16.
 * Boxes are processed in chunks that fit the workspace.  A network whose
 * per-box workspace exceeds 32 MiB, or whose tables exceed 4 MiB, is rejected
 * with BERN_E_UNSUPPORTED before any GPU work.
 * The first call on a device (the current device) looks up the addresses of
 * the static arrays and uploads the tables; make that first call before any
 * stream capture.  The call synchronises `stream` at its end and returns the
 * device-side status like bern_sync.  All calls share the one workspace:
 * calls that overlap on the GPU (other streams or threads) race and must be
 * serialised by the caller. */
int bern_propagate_noalloc(const bern_net* net, const float* boxes, int64_t n_boxes,
                           const bern_degree_plan* plan, bern_result* result, void* stream);

/* ------------------------------------------------------------ learned component
 * The proposals only choose orders; bern_propagate computes sound bounds for
 * whatever order it is given, so the MLP never affects soundness. */

/* Features of n_boxes boxes for split-dimension proposals (2n + 2 per box,
 * so n <= 7 for a BERN_MLP_MAX_FEATURES input), from the boxes, the root
 * box the search started from, and a bern_result of those boxes (device
 * pointers, coef required), for output j:  with c_up / c_lo the output's
 * upper / lower polynomial and e_k(r) the exponent of t_k in monomial r,
 *   x[k]      = log2(side_k / root_side_k) / 16              (k < n)
 *   x[n + k]  = s_k / sum_i s_i,  s_k = sum_r |c_up_r| e_k(r)  (k < n)
 *   x[2n]     = log2(max(hi_j - lo_j, 1e-30)) / 8
 *   x[2n + 1] = log2(max(sum_r |c_up_r - c_lo_r|, 1e-30)) / 8
 * x: [n_boxes x (2n + 2)] fp32. */
int bern_split_features(bern_ctx* ctx, int n, int64_t n_boxes, const float* boxes,
                        const float* root_box, const bern_result* result, int n_outputs,
                        int output, float* x);

/* Number of FP32 parameters of an MLP (W1, b1, W2, b2). */
int64_t bern_mlp_num_params(int n_features, int n_classes);

/* Features of n_items (box, neuron) items for degree proposals, from the
 * pre-activation enclosure [lo, hi], the pre-activation term count and the
 * hidden layer index (1-based):  with s = max(|lo|, |hi|, 1e-30),
 *   x0 = lo/s, x1 = hi/s, x2 = log2(max(hi-lo, 1e-30))/8, x3 = layer/8,
 *   x4 = log2(max(nterms, 1))/16, x5 = [lo >= 0], x6 = [hi <= 0],
 *   x7 = -lo/(hi-lo) clipped to [0, 1] (the kink position, 0 if lo >= 0).
 * x: [n_items x BERN_DEGREE_FEATURES] fp32. */
int bern_degree_features(bern_ctx* ctx, int64_t n_items, const float* lo, const float* hi,
                         const int32_t* nterms, int layer, float* x);

/* Inference: logits [n x n_classes] fp32 for features x [n x n_features]. */
int bern_mlp_forward(bern_ctx* ctx, const bern_mlp* mlp, int64_t n, const float* x,
                     float* logits);

/* Training step, part 1: the gradient of the mean weighted softmax
 * cross-entropy  L = (1/n) sum_s w_s * (-log softmax(z_s)[label_s])
 * with respect to the flat parameter vector (W1, b1, W2, b2), through the
 * BF16 forward above (the bf16 roundings of x and a are treated as the
 * identity in the derivative).  labels: [n] int32 in [0, n_classes);
 * w: [n] fp32 or NULL (all 1).  grad: [num_params] fp32, loss: [1] fp32.
 * Deterministic (fixed summation order).  Uses library scratch. */
int bern_mlp_backward(bern_ctx* ctx, const bern_mlp* mlp, int64_t n, const float* x,
                      const int32_t* labels, const float* w, float* grad, float* loss);

/* Training step, part 2: one Adam update (Kingma & Ba, with bias
 * correction for step t >= 1) of the FP32 master parameters `param`
 * (with moments m, v, all [num_params]), then the BF16 copies of W1 and W2
 * (round to nearest even) into W1_bf16 / W2_bf16. */
int bern_mlp_adam(bern_ctx* ctx, int n_features, int n_classes, float* param, float* m,
                  float* v, const float* grad, float lr, float beta1, float beta2, float eps,
                  int t, uint16_t* W1_bf16, uint16_t* W2_bf16);

#ifdef __cplusplus
}
#endif
#endif /* BERN_H */
