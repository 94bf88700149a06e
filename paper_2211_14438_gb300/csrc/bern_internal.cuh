// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
// Same for the product of a degree-Dq polynomial by a degree-Ds one:
// pairs (I in q, J in s), packed I | (J << 16)
bool build_product_pairs(int n, int Dq, int Ds, PairList& out);

// ------------------------------------------------------------ device views
struct PairTable {
  const int32_t* ptr;
  const uint32_t* pairs;
};

struct Tables {
  int n;
  int dmax;                        // degrees 0..dmax have square tables
  const uint8_t* exps;             // graded exponents, mexps ranks
  int64_t mexps;
  const int32_t* mcount;           // M(n, D) for D = 0..64
  PairTable sq[kMaxTableDegree + 1];
  // rscale[l][r]: float bracket (lo, hi) of 1 / prod_k C(l, e_k(r)) for the
  // ranks r < M(n, l), for Bernstein orders l = 0..rscale_max
  const float2* rscale[kMaxEncloseOrder + 1];
  int rscale_max;
};

// Largest Bernstein order whose grid fits the shared-memory limit for n vars.
int max_enclose_order(int n);
// Host image of the reciprocal brackets for order l: 2*M(n,l) floats.
void build_rscale(int n, int l, std::vector<float>& out);

// ------------------------------------------------------------ launchers
struct Launch {
  cudaStream_t stream;
  int* status;                     // device status word
  int64_t* launches;               // host counter
};

cudaError_t launch_init_inputs(const Launch& L, int n, int64_t n_boxes, const float* boxes,
                               float* z_up, float* z_lo, int64_t stride, int32_t* nterms);
cudaError_t launch_affine(const Launch& L, int64_t n_boxes, int h_out, int h_in,
                          const float* W, const float* b, const float* in_up,
                          const float* in_lo, int64_t in_stride, const int32_t* in_nterms,
                          float* out_up, float* out_lo, int64_t out_stride,
                          int32_t* out_nterms);
cudaError_t launch_enclose(const Launch& L, const Tables& T, int64_t n_items, int order,
                           int64_t budget, const float* pre_up, const float* pre_lo,
                           int64_t stride, const int32_t* nterms, float* lo, float* hi);
cudaError_t launch_enclose_relu(const Launch& L, const Tables& T, int64_t n_items, int order,
                                int64_t budget, const float* pre_up, const float* pre_lo,
                                int64_t stride, const int32_t* nterms, float* lo, float* hi,
                                const uint8_t* degrees, int global_d, int8_t* kind, float* coef,
                                float* eps);
cudaError_t launch_relu_coeffs(const Launch& L, int64_t n_items, const float* lo,
                               const float* hi, const uint8_t* degrees, int global_d,
                               int8_t* kind, float* coef, float* eps);
cudaError_t launch_compose(const Launch& L, const Tables& T, int64_t n_items, int cap,
                           float tau, const int8_t* kind, const float* coef,
                           const float* eps, const uint8_t* degrees, int global_d,
                           const float* lo, const float* hi, const float* pre_up,
                           const float* pre_lo, int64_t pre_stride,
                           const int32_t* pre_nterms, float* post_up, float* post_lo,
                           int64_t post_stride, int32_t* post_nterms);
cudaError_t launch_pack(const Launch& L, const Tables& T, int64_t n_boxes, int o,
                        const float* pre_up, const float* pre_lo, int64_t stride,
                        const int32_t* nterms, bern_result res);

}  // namespace bern
