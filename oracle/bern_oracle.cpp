// BERN-NN reference oracle: plain, slow, FP64, single-threaded.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
// load this file; only the test suite, the smoke check and the CPU-baseline
// leg of the benchmark use it.  It shares no header, table or helper with the
// CUDA library.
//
// What it computes (arxiv 2211.14438, "BERN-NN"):
//   Problem 1 (Sec. 2): polynomials p_lo(x) <= NN_j(x) <= p_up(x) on a box.
//   Layer step (Sec. 5.2, eqs. upper_bounds_layer / lower_bounds_layer):
//       up' = W+ up + W- lo + b,   lo' = W+ lo + W- up + b.
//   Step 1 (Sec. 5.1, eq. find_lo_hi): lo = min of the Bernstein coefficients
//       of the lower pre-activation polynomial, hi = max of those of the upper
//       one (range enclosing property, Def. 2).
//   Step 2 (Sec. 5.1): the order-L Bernstein polynomial of ReLU on [lo,hi]
//       (Def. 1, Prop. 1) in power form; its maximal error is its value at 0
//       (Prop. 2, eq. max_error), so the under-approximation is the same
//       polynomial shifted down by that value.
//   Step 3 (Sec. 5.1, eqs. post_bounds_1/2): compose the over-approximation
//       with the upper and the shifted one with the lower pre-activation.
//   Input init (Sec. 5.3): z0_i = x_i on the box.
//
// Readings where the paper is silent (numbered as in the design notes):
//   * Polynomials are stored in the power basis of the normalised variables
//     t_i = (x_i - dlo_i)/(dhi_i - dlo_i) in [0,1]; Bernstein coefficients are
//     formed only inside the enclosure.  (R1)
//   * Def. 2 refers to the exact Bernstein expansion of the polynomial
//     (p == sum_I b_I Ber_I), whose coefficients on [0,1]^n are
//     b_I = sum_{J<=I} prod_k C(i_k,j_k)/C(l_k,j_k) a_J.  Def. 1's samples of
//     p at grid points would not bound p.  (R15)
//   * The Bernstein order used by the enclosure at layer i is the paper's own
//     order bookkeeping L_z = L_zhat * L (Sec. 5.1), starting from order 1 at
//     the input (Sec. 5.3), capped at the total-degree cap.  (R3/R6)
//   * A neuron with hi <= 0 outputs 0 and one with lo >= 0 passes its input
//     through; in exact arithmetic this equals the Bernstein formulas,
//     because Bernstein polynomials reproduce linear functions.  (R2)
//   * Power form of the ReLU polynomial is taken in s = (y-lo)/(hi-lo), an
//     affine change of variable that leaves the composition unchanged.  (R9)
//   * Terms of total degree above the cap, and (tau > 0) terms with
//     |c| < tau*||q||_1, are dropped after every product in the Horner
//     evaluation; each dropped term c t^K lies in [min(0,c), max(0,c)] on
//     the box, so the upper chain adds max(0,c) and the lower chain min(0,c)
//     to a one-sided remainder; the remainder r is carried through each
//     further product by s in [0,1] as max(0,r) (upper) or min(0,r) (lower),
//     and finally added to the constant term.  (R4/R5)
//   * If the Bernstein grid (l+1)^n exceeds the budget, the enclosure uses
//     the largest order l' with (l'+1)^n <= budget for the terms of total
//     degree <= l' and the interval [min(0,c),max(0,c)] for every other
//     term.  (R6)
//   * Lin (Sec. 5.3): every Lin hidden layers the post-activation bounds are
//     lowered to order [1,...,1], i.e. to multilinear polynomials.  The cited
//     linearisation algorithm is not given; here A is the least-squares fit of
//     P on the box (the multilinear polynomial minimising the integral of
//     (P - A)^2 over [0,1]^n), the residual P - A is enclosed by its Bernstein
//     coefficients at the layer's order (Def. 2), and the bound becomes A plus
//     the residual's max (upper) or min (lower).  The shift makes the result
//     sound for any A; the fit only decides how tight it is.  The next
//     layer's order is then min(n, order): the total degree of a multilinear
//     polynomial of total degree <= order.  (R22)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <vector>

namespace {

typedef std::vector<int> Mono;            // exponent vector, one entry per t_k
typedef std::map<Mono, double> Poly;      // sum_K a_K t^K

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return std::round(r);
}

int total_degree(const Mono& m) {
  int s = 0;
  for (int e : m) s += e;
  return s;
}

Poly poly_const(int n, double c) {
  Poly p;
  p[Mono(n, 0)] = c;
  return p;
}

void add_to(Poly& p, const Mono& k, double c) { p[k] += c; }

// p*q: every pair of terms, exponents added (the power-series product Prod,
// Sec. 4.2).
Poly poly_mul(const Poly& p, const Poly& q) {
  Poly r;
  for (const auto& a : p)
    for (const auto& b : q) {
      Mono k(a.first.size());
      for (size_t i = 0; i < k.size(); ++i) k[i] = a.first[i] + b.first[i];
      r[k] += a.second * b.second;
    }
  return r;
}

// ---------------------------------------------------------------- enclosure
// Bernstein coefficients of p on [0,1]^n, order l in every variable, indexed
// in mixed radix (l+1) with t_1 the slowest digit.
bool bernstein_coeffs(const Poly& p, int n, int l, std::vector<double>& out) {
  size_t grid = 1;
  for (int k = 0; k < n; ++k) grid *= (size_t)(l + 1);
  out.assign(grid, 0.0);
  for (const auto& term : p)
    for (int k = 0; k < n; ++k)
      if (term.first[k] > l) return false;
  std::vector<int> I(n, 0);
  for (size_t g = 0; g < grid; ++g) {
    size_t rem = g;
    for (int k = n - 1; k >= 0; --k) {
      I[k] = (int)(rem % (size_t)(l + 1));
      rem /= (size_t)(l + 1);
    }
    double b = 0.0;
    for (const auto& term : p) {
      const Mono& J = term.first;
      double w = 1.0;
      for (int k = 0; k < n && w != 0.0; ++k)
        w *= binom(I[k], J[k]) / binom(l, J[k]);   // zero unless J_k <= I_k
      b += w * term.second;
    }
    out[g] = b;
  }
  return true;
}

// The same coefficients with the weight's factorisation over the variables:
// prod_k C(i_k, j_k) / C(l, j_k) = prod_k C(i_k, j_k) * (1 / prod_k C(l, j_k)),
// so b = T_1 (x) ... (x) T_n applied to c_J = a_J / prod_k C(l, j_k), where T
// is the lower-triangular matrix C(i, j), j <= i <= l.  Applied one variable
// at a time (line by line), that is n (l+1)^n (l+2)/2 multiply-adds instead of
// (l+1)^n times the number of terms; used for large grids.
bool bernstein_coeffs_factored(const Poly& p, int n, int l, std::vector<double>& out) {
  const size_t R = (size_t)(l + 1);
  size_t grid = 1;
  for (int k = 0; k < n; ++k) grid *= R;
  out.assign(grid, 0.0);
  for (const auto& term : p) {
    size_t idx = 0;
    double scale = 1.0;
    for (int k = 0; k < n; ++k) {
      if (term.first[k] > l) return false;
      idx = idx * R + (size_t)term.first[k];
      scale *= binom(l, term.first[k]);
    }
    out[idx] += term.second / scale;
  }
  std::vector<double> x(R), y(R);
  for (int k = 0; k < n; ++k) {
    size_t stride = 1;
    for (int m = k + 1; m < n; ++m) stride *= R;
    // every line along variable k: cells whose digit k runs over 0..l
    for (size_t g = 0; g < grid; ++g) {
      if ((g / stride) % R != 0) continue;      // g is the line's first cell
      for (size_t i = 0; i < R; ++i) x[i] = out[g + i * stride];
      for (size_t i = 0; i < R; ++i) {
        double acc = 0.0;
        for (size_t j = 0; j <= i; ++j) acc += binom((int)i, (int)j) * x[j];
        y[i] = acc;
      }
      for (size_t i = 0; i < R; ++i) out[g + i * stride] = y[i];
    }
  }
  return true;
}

size_t grid_size(int n, int l) {
  size_t g = 1;
  for (int k = 0; k < n; ++k) {
    g *= (size_t)(l + 1);
    if (g > ((size_t)1 << 40)) return g;
  }
  return g;
}

// Enclosure [emin, emax] of p on [0,1]^n (Def. 2), with the budget rule.
bool enclosure(const Poly& p, int n, int l, long long budget, double* emin,
               double* emax) {
  int lb = l;
  if (budget > 0)
    while (lb > 0 && grid_size(n, lb) > (size_t)budget) --lb;
  Poly head;
  double rlo = 0.0, rhi = 0.0;
  for (const auto& t : p) {
    if (total_degree(t.first) <= lb) {
      head[t.first] += t.second;
    } else {
      rlo += std::min(0.0, t.second);
      rhi += std::max(0.0, t.second);
    }
  }
  if (head.empty()) head = poly_const(n, 0.0);
  std::vector<double> b;
  // the definition term by term while it is cheap, the factored form above
  if ((double)grid_size(n, lb) * (double)head.size() <= 4.0e6) {
    if (!bernstein_coeffs(head, n, lb, b)) return false;
  } else {
    if (!bernstein_coeffs_factored(head, n, lb, b)) return false;
  }
  double mn = b[0], mx = b[0];
  for (double v : b) {
    mn = std::min(mn, v);
    mx = std::max(mx, v);
  }
  *emin = mn + rlo;
  *emax = mx + rhi;
  return true;
}

// ----------------------------------------------------------------- ReLU step
// Def. 1 applied to sigma(y) = max(0,y) on [lo,hi], order d, univariate.
double relu_bern_eval(double lo, double hi, int d, double y) {
  double s = (y - lo) / (hi - lo);
  double v = 0.0;
  for (int k = 0; k <= d; ++k) {
    double node = lo + (hi - lo) * k / d;
    double bk = node > 0.0 ? node : 0.0;
    v += bk * binom(d, k) * std::pow(s, k) * std::pow(1.0 - s, d - k);
  }
  return v;
}

// Power form in s of the order-d Bernstein polynomial of ReLU on [lo,hi]:
// expand each basis term C(d,k) s^k (1-s)^(d-k) by the binomial theorem.
// eps = value of the polynomial at y = 0 (Prop. 2).
void relu_coeffs(double lo, double hi, int d, double* a, double* eps) {
  for (int j = 0; j <= d; ++j) a[j] = 0.0;
  for (int k = 0; k <= d; ++k) {
    double node = lo + (hi - lo) * k / d;
    double bk = node > 0.0 ? node : 0.0;
    for (int m = 0; m <= d - k; ++m) {
      double sign = (m % 2) ? -1.0 : 1.0;
      a[k + m] += bk * binom(d, k) * binom(d - k, m) * sign;
    }
  }
  *eps = relu_bern_eval(lo, hi, d, 0.0);
}

// ---------------------------------------------------------------- Step 3
// One bound of one neuron: B(s(t)) with s = (P - lo)/(hi - lo), by Horner in
// the power form a_j, truncating at the cap (and pruning) after each product.
Poly compose(const Poly& P, int n, double lo, double hi, const double* a, int d,
             double eps, int cap, double tau, bool upper) {
  Poly s;
  for (const auto& t : P) s[t.first] = t.second / (hi - lo);
  s[Mono(n, 0)] += -lo / (hi - lo);
  Poly q = poly_const(n, a[d]);
  double r = 0.0;
  for (int j = d - 1; j >= 0; --j) {
    q = poly_mul(q, s);
    r = upper ? std::max(0.0, r) : std::min(0.0, r);
    q[Mono(n, 0)] += a[j];
    for (auto it = q.begin(); it != q.end();) {
      if (total_degree(it->first) > cap) {
        r += upper ? std::max(0.0, it->second) : std::min(0.0, it->second);
        it = q.erase(it);
      } else {
        ++it;
      }
    }
    if (tau > 0.0) {
      double norm = 0.0;
      for (const auto& t : q) norm += std::fabs(t.second);
      for (auto it = q.begin(); it != q.end();) {
        if (total_degree(it->first) > 0 && std::fabs(it->second) < tau * norm) {
          r += upper ? std::max(0.0, it->second) : std::min(0.0, it->second);
          it = q.erase(it);
        } else {
          ++it;
        }
      }
    }
  }
  q[Mono(n, 0)] += r;
  if (!upper) q[Mono(n, 0)] -= eps;
  return q;
}

// Affine step of Sec. 5.2 for all neurons of one layer.
void affine(const std::vector<Poly>& up, const std::vector<Poly>& lo,
            const double* W, const double* b, int h_out, int h_in, int n,
            std::vector<Poly>& pre_up, std::vector<Poly>& pre_lo) {
  pre_up.assign(h_out, Poly());
  pre_lo.assign(h_out, Poly());
  for (int m = 0; m < h_out; ++m) {
    Poly pu = poly_const(n, b[m]);
    Poly pl = poly_const(n, b[m]);
    for (int j = 0; j < h_in; ++j) {
      double w = W[(size_t)m * h_in + j];
      double wp = w > 0.0 ? w : 0.0;     // W+
      double wn = w < 0.0 ? w : 0.0;     // W-
      for (const auto& t : up[j]) {
        pu[t.first] += wp * t.second;
        pl[t.first] += wn * t.second;
      }
      for (const auto& t : lo[j]) {
        pu[t.first] += wn * t.second;
        pl[t.first] += wp * t.second;
      }
    }
    pre_up[m] = pu;
    pre_lo[m] = pl;
  }
}

Poly from_arrays(int n, int nterms, const uint8_t* exps, const double* coef) {
  Poly p;
  for (int i = 0; i < nterms; ++i) {
    Mono k(n);
    for (int v = 0; v < n; ++v) k[v] = exps[(size_t)i * n + v];
    p[k] += coef[i];
  }
  return p;
}

int to_arrays(const Poly& p, int n, int cap_terms, int* nterms, uint8_t* exps,
              double* coef) {
  *nterms = (int)p.size();
  if ((int)p.size() > cap_terms) return 2;
  int i = 0;
  for (const auto& t : p) {
    for (int v = 0; v < n; ++v) exps[(size_t)i * n + v] = (uint8_t)t.first[v];
    coef[i] = t.second;
    ++i;
  }
  return 0;
}

// ------------------------------------------------------------- Lin step
// The least-squares fit is the solution of its normal equations, written out:
// over the multilinear monomials t^S (S a set of variables, |S| <= min(n, deg P);
// the fit of a degree-D polynomial has degree <= D) the Gram matrix is
// G_ST = integral of t^S t^T = prod_k 1/(s_k + t_k + 1) and the right-hand side
// m_S = integral of P t^S = sum_K p_K prod_k 1/(k_k + s_k + 1); solved by
// Gaussian elimination with partial pivoting.
bool linearize(const Poly& P, int n, int order, long long budget, bool upper, Poly& out) {
  int D = 0;
  for (const auto& t : P) D = std::max(D, total_degree(t.first));
  const int Dl = std::min(n, D);
  std::vector<Mono> basis;
  for (int s = 0; s < (1 << n); ++s) {
    Mono S(n, 0);
    int c = 0;
    for (int k = 0; k < n; ++k)
      if ((s >> k) & 1) {
        S[k] = 1;
        ++c;
      }
    if (c <= Dl) basis.push_back(S);
  }
  const size_t N = basis.size();
  std::vector<double> G(N * N), rhs(N), a(N);
  for (size_t i = 0; i < N; ++i) {
    for (size_t j = 0; j < N; ++j) {
      double g = 1.0;
      for (int k = 0; k < n; ++k) g /= (double)(basis[i][k] + basis[j][k] + 1);
      G[i * N + j] = g;
    }
    double m = 0.0;
    for (const auto& t : P) {
      double w = 1.0;
      for (int k = 0; k < n; ++k) w /= (double)(t.first[k] + basis[i][k] + 1);
      m += t.second * w;
    }
    rhs[i] = m;
  }
  for (size_t col = 0; col < N; ++col) {
    size_t piv = col;
    for (size_t r = col + 1; r < N; ++r)
      if (std::fabs(G[r * N + col]) > std::fabs(G[piv * N + col])) piv = r;
    if (G[piv * N + col] == 0.0) return false;
    if (piv != col) {
      for (size_t c = 0; c < N; ++c) std::swap(G[piv * N + c], G[col * N + c]);
      std::swap(rhs[piv], rhs[col]);
    }
    for (size_t r = col + 1; r < N; ++r) {
      const double f = G[r * N + col] / G[col * N + col];
      for (size_t c = col; c < N; ++c) G[r * N + c] -= f * G[col * N + c];
      rhs[r] -= f * rhs[col];
    }
  }
  for (size_t i = N; i-- > 0;) {
    double v = rhs[i];
    for (size_t j = i + 1; j < N; ++j) v -= G[i * N + j] * a[j];
    a[i] = v / G[i * N + i];
  }
  Poly A;
  for (size_t i = 0; i < N; ++i) A[basis[i]] = a[i];
  Poly R = P;
  for (const auto& t : A) R[t.first] -= t.second;
  double emin, emax;
  if (!enclosure(R, n, order, budget, &emin, &emax)) return false;
  A[Mono(n, 0)] += upper ? emax : emin;
  out = A;
  return true;
}

}  // namespace

extern "C" {

double orc_binom(int n, int k) { return binom(n, k); }

double orc_relu_bern_eval(double lo, double hi, int d, double y) {
  return relu_bern_eval(lo, hi, d, y);
}

void orc_relu_coeffs(double lo, double hi, int d, double* a, double* eps) {
  relu_coeffs(lo, hi, d, a, eps);
}

// Bernstein coefficients (order l in every variable) of a polynomial given by
// nterms (exponent row, coefficient) pairs.  out has (l+1)^n entries.
int orc_bernstein_coeffs(int n, int nterms, const uint8_t* exps,
                         const double* coef, int l, double* out) {
  std::vector<double> b;
  if (!bernstein_coeffs(from_arrays(n, nterms, exps, coef), n, l, b)) return 1;
  std::memcpy(out, b.data(), b.size() * sizeof(double));
  return 0;
}

int orc_bernstein_coeffs_factored(int n, int nterms, const uint8_t* exps,
                                  const double* coef, int l, double* out) {
  std::vector<double> b;
  if (!bernstein_coeffs_factored(from_arrays(n, nterms, exps, coef), n, l, b)) return 1;
  std::memcpy(out, b.data(), b.size() * sizeof(double));
  return 0;
}

int orc_enclosure(int n, int nterms, const uint8_t* exps, const double* coef,
                  int l, long long budget, double* emin, double* emax) {
  return enclosure(from_arrays(n, nterms, exps, coef), n, l, budget, emin, emax)
             ? 0 : 1;
}

int orc_compose(int n, int nterms, const uint8_t* exps, const double* coef,
                double lo, double hi, int d, int cap, double tau, int upper,
                int cap_terms, int* out_n, uint8_t* out_exps, double* out_coef) {
  std::vector<double> a(d + 1);
  double eps;
  relu_coeffs(lo, hi, d, a.data(), &eps);
  Poly q = compose(from_arrays(n, nterms, exps, coef), n, lo, hi, a.data(), d,
                   eps, cap, tau, upper != 0);
  return to_arrays(q, n, cap_terms, out_n, out_exps, out_coef);
}

int orc_poly_mul(int n, int na, const uint8_t* ea, const double* ca, int nb,
                 const uint8_t* eb, const double* cb, int cap_terms, int* out_n,
                 uint8_t* out_exps, double* out_coef) {
  Poly r = poly_mul(from_arrays(n, na, ea, ca), from_arrays(n, nb, eb, cb));
  return to_arrays(r, n, cap_terms, out_n, out_exps, out_coef);
}

// Affine step (Sec. 5.2) for one output neuron: h_in upper/lower input
// polynomials given back to back (nterms per polynomial in nt_up/nt_lo).
int orc_affine(int n, int h_in, const int* nt_up, const uint8_t* e_up,
               const double* c_up, const int* nt_lo, const uint8_t* e_lo,
               const double* c_lo, const double* w_row, double bias, int cap_terms,
               int* out_n, uint8_t* out_exps, double* out_coef) {
  std::vector<Poly> up(h_in), lo(h_in);
  size_t ou = 0, ol = 0;
  for (int j = 0; j < h_in; ++j) {
    up[j] = from_arrays(n, nt_up[j], e_up + ou * n, c_up + ou);
    lo[j] = from_arrays(n, nt_lo[j], e_lo + ol * n, c_lo + ol);
    ou += nt_up[j];
    ol += nt_lo[j];
  }
  std::vector<Poly> pu, pl;
  affine(up, lo, w_row, &bias, 1, h_in, n, pu, pl);
  int rc = to_arrays(pu[0], n, cap_terms, &out_n[0], out_exps, out_coef);
  int rc2 = to_arrays(pl[0], n, cap_terms, &out_n[1], out_exps + (size_t)cap_terms * n,
                      out_coef + cap_terms);
  return rc ? rc : rc2;
}

// Lin step on one polynomial (upper != 0: the upper bound's shift).
int orc_linearize(int n, int nterms, const uint8_t* exps, const double* coef, int order,
                  long long budget, int upper, int cap_terms, int* out_n, uint8_t* out_exps,
                  double* out_coef) {
  Poly out;
  if (!linearize(from_arrays(n, nterms, exps, coef), n, order, budget, upper != 0, out))
    return 1;
  return to_arrays(out, n, cap_terms, out_n, out_exps, out_coef);
}

void orc_eval_poly(int n, int nterms, const uint8_t* exps, const double* coef,
                   long long npts, const double* t, double* out) {
  for (long long p = 0; p < npts; ++p) {
    double v = 0.0;
    for (int i = 0; i < nterms; ++i) {
      double m = coef[i];
      for (int k = 0; k < n; ++k) {
        int e = exps[(size_t)i * n + k];
        for (int r = 0; r < e; ++r) m *= t[(size_t)p * n + k];
      }
      v += m;
    }
    out[p] = v;
  }
}

// Whole network, one box.
//   widths[0..H]; W_all/b_all: the layers' row-major weights and biases back
//   to back; box: n (lo,hi) pairs; degrees: ReLU order per hidden neuron
//   (sum of hidden widths entries, layer-major); lin: linearise the
//   post-activation bounds after every lin-th hidden layer (0: never).
//   Outputs: out_lo/out_hi (o), out_nterms (o x 2: upper, lower),
//   out_exps (o x 2 x cap_terms x n), out_coef (o x 2 x cap_terms);
//   trace arrays per hidden neuron: lo, hi, case (0 dead, 1 pass, 2 relu),
//   and per layer (H entries) the Bernstein order used by the enclosure.
// Returns 0, 1 (order exceeds grid), 2 (output capacity too small),
// 3 (invalid input).
}  // extern "C"

namespace {

// Choice of the ReLU order of hidden neuron m of hidden layer `layer`
// (1-based; hidden_idx counts hidden neurons layer-major) from its
// pre-activation enclosure and the dense term count M(n, D) of its
// pre-activation polynomials (D = their largest total degree).
using DegreeChoice = std::function<int(int layer, int m, int hidden_idx, double lo, double hi,
                                       long long nterms)>;

long long dense_terms(const Poly& p, int n) {
  int D = 0;
  for (const auto& t : p) D = std::max(D, total_degree(t.first));
  double m = 1.0;
  for (int i = 1; i <= n; ++i) m = m * (double)(D + i) / (double)i;
  return (long long)std::llround(m);
}

int propagate_core(int H, const int* widths, const double* W_all,
                   const double* b_all, const double* box, const DegreeChoice& choose,
                   int cap, double tau, long long budget, int lin, double* out_lo,
                   double* out_hi, int cap_terms, int* out_nterms,
                   uint8_t* out_exps, double* out_coef, double* tr_lo,
                   double* tr_hi, int* tr_case, int* tr_order, int* tr_degree) {
  const int n = widths[0];
  if (H < 1 || n < 1 || n > 8 || cap < 1) return 3;
  std::vector<Poly> up(n), lo(n);
  for (int i = 0; i < n; ++i) {
    double dl = box[2 * i], dh = box[2 * i + 1];
    if (!(dl <= dh)) return 3;
    Poly x = poly_const(n, dl);
    Mono k(n, 0);
    k[i] = 1;
    x[k] = dh - dl;
    up[i] = x;
    lo[i] = x;
  }
  size_t woff = 0, boff = 0;
  int order = 1;
  int hidden_idx = 0;
  for (int layer = 1; layer <= H; ++layer) {
    int h_in = widths[layer - 1], h_out = widths[layer];
    std::vector<Poly> pu, pl;
    affine(up, lo, W_all + woff, b_all + boff, h_out, h_in, n, pu, pl);
    woff += (size_t)h_out * h_in;
    boff += (size_t)h_out;
    tr_order[layer - 1] = order;
    if (layer == H) {
      for (int m = 0; m < h_out; ++m) {
        double emin, emax, dummy;
        if (!enclosure(pl[m], n, order, budget, &emin, &dummy)) return 1;
        if (!enclosure(pu[m], n, order, budget, &dummy, &emax)) return 1;
        out_lo[m] = emin;
        out_hi[m] = emax;
        size_t base = (size_t)m * 2;
        int rc = to_arrays(pu[m], n, cap_terms, &out_nterms[base],
                           out_exps + base * cap_terms * n,
                           out_coef + base * cap_terms);
        int rc2 = to_arrays(pl[m], n, cap_terms, &out_nterms[base + 1],
                            out_exps + (base + 1) * cap_terms * n,
                            out_coef + (base + 1) * cap_terms);
        if (rc || rc2) return 2;
      }
      break;
    }
    std::vector<Poly> nu(h_out), nl(h_out);
    int dmax = 1;
    for (int m = 0; m < h_out; ++m) {
      double lom, him, dummy;
      if (!enclosure(pl[m], n, order, budget, &lom, &dummy)) return 1;
      if (!enclosure(pu[m], n, order, budget, &dummy, &him)) return 1;
      int d = choose(layer, m, hidden_idx, lom, him, dense_terms(pu[m], n));
      if (d < 1) return 3;
      if (tr_degree) tr_degree[hidden_idx] = d;
      dmax = std::max(dmax, d);
      tr_lo[hidden_idx] = lom;
      tr_hi[hidden_idx] = him;
      if (him <= 0.0) {
        tr_case[hidden_idx] = 0;
        nu[m] = poly_const(n, 0.0);
        nl[m] = poly_const(n, 0.0);
      } else if (lom >= 0.0) {
        tr_case[hidden_idx] = 1;
        nu[m] = pu[m];
        nl[m] = pl[m];
      } else {
        tr_case[hidden_idx] = 2;
        std::vector<double> a(d + 1);
        double eps;
        relu_coeffs(lom, him, d, a.data(), &eps);
        nu[m] = compose(pu[m], n, lom, him, a.data(), d, eps, cap, tau, true);
        nl[m] = compose(pl[m], n, lom, him, a.data(), d, eps, cap, tau, false);
      }
      ++hidden_idx;
    }
    order = std::min(order * dmax, cap);
    if (lin > 0 && layer % lin == 0) {
      for (int m = 0; m < h_out; ++m) {
        Poly a, c;
        if (!linearize(nu[m], n, order, budget, true, a)) return 1;
        if (!linearize(nl[m], n, order, budget, false, c)) return 1;
        nu[m] = a;
        nl[m] = c;
      }
      order = std::min(n, order);
    }
    up.swap(nu);
    lo.swap(nl);
  }
  return 0;
}

}  // namespace

extern "C" {

int orc_propagate(int H, const int* widths, const double* W_all,
                  const double* b_all, const double* box, const int* degrees,
                  int cap, double tau, long long budget, int lin, double* out_lo,
                  double* out_hi, int cap_terms, int* out_nterms,
                  uint8_t* out_exps, double* out_coef, double* tr_lo,
                  double* tr_hi, int* tr_case, int* tr_order) {
  DegreeChoice fixed = [degrees](int, int, int k, double, double, long long) {
    return degrees[k];
  };
  return propagate_core(H, widths, W_all, b_all, box, fixed, cap, tau, budget, lin, out_lo, out_hi,
                        cap_terms, out_nterms, out_exps, out_coef, tr_lo, tr_hi, tr_case,
                        tr_order, nullptr);
}

// Same, with the order of every hidden neuron chosen at run time by a
// callback (the learned component's proposals); the chosen orders are
// written to tr_degree.
typedef int (*orc_degree_fn)(void* user, int layer, int m, double lo, double hi,
                             long long nterms);
int orc_propagate_cb(int H, const int* widths, const double* W_all,
                     const double* b_all, const double* box, orc_degree_fn fn, void* user,
                     int cap, double tau, long long budget, int lin, double* out_lo,
                     double* out_hi, int cap_terms, int* out_nterms,
                     uint8_t* out_exps, double* out_coef, double* tr_lo,
                     double* tr_hi, int* tr_case, int* tr_order, int* tr_degree) {
  DegreeChoice cb = [fn, user](int layer, int m, int, double lo, double hi, long long nt) {
    return fn(user, layer, m, lo, hi, nt);
  };
  return propagate_core(H, widths, W_all, b_all, box, cb, cap, tau, budget, lin, out_lo, out_hi,
                        cap_terms, out_nterms, out_exps, out_coef, tr_lo, tr_hi, tr_case,
                        tr_order, tr_degree);
}

}  // extern "C"
