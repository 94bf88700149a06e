// Host-side monomial tables: the graded order and the pair lists that drive
// the composition kernel's polynomial products (the power-series product
// "Prod" of Sec. 4.2, here over a shared dense graded monomial set).
#include <algorithm>
#include <cmath>
#include <unordered_map>

#include "bern_internal.cuh"

namespace bern {

int64_t num_monomials(int n, int D) {
  if (n < 1 || n > kMaxVars || D < 0 || D > kMaxTableDegree) return -1;
  // C(n+D, n) by the multiplicative formula (exact in 64 bits here)
  unsigned __int128 r = 1;
  for (int i = 1; i <= n; ++i) r = r * (unsigned)(D + i) / (unsigned)i;
  return (int64_t)r;
}

uint64_t pack_key(const uint8_t* e, int n) {
  uint64_t k = 0;
  for (int i = 0; i < n; ++i) k |= (uint64_t)e[i] << (8 * i);
  return k;
}

// all exponent vectors of n variables with sum g, descending lexicographic
static void rec(int n, int pos, int left, std::vector<uint8_t>& cur,
                std::vector<uint8_t>& out) {
  if (pos == n - 1) {
    cur[pos] = (uint8_t)left;
    out.insert(out.end(), cur.begin(), cur.end());
    return;
  }
  for (int e = left; e >= 0; --e) {
    cur[pos] = (uint8_t)e;
    rec(n, pos + 1, left - e, cur, out);
  }
}

void graded_monomials(int n, int D, std::vector<uint8_t>& exps) {
  exps.clear();
  std::vector<uint8_t> cur(n, 0);
  for (int g = 0; g <= D; ++g) rec(n, 0, g, cur, exps);
}

static bool build_pairs(int n, int Dq, int Ds, bool symmetric, PairList& out) {
  const int64_t mq = num_monomials(n, Dq), ms = num_monomials(n, Ds);
  const int64_t mo = num_monomials(n, Dq + Ds);
  if (mq < 0 || ms < 0 || mo < 0 || mq > 65535 || ms > 65535) return false;
  if (mo > (int64_t)1 << 30) return false;
  std::vector<uint8_t> ex;
  graded_monomials(n, Dq + Ds, ex);
  std::unordered_map<uint64_t, int32_t> rank;
  rank.reserve((size_t)mo * 2);
  for (int64_t r = 0; r < mo; ++r) rank[pack_key(&ex[(size_t)r * n], n)] = (int32_t)r;
  std::vector<uint64_t> kq(mq), ks(ms);
  for (int64_t r = 0; r < mq; ++r) kq[r] = pack_key(&ex[(size_t)r * n], n);
  for (int64_t r = 0; r < ms; ++r) ks[r] = pack_key(&ex[(size_t)r * n], n);
  // exponents are < 256 in every slot, so key addition never carries
  std::vector<int32_t> cnt(mo + 1, 0);
  for (int64_t i = 0; i < mq; ++i)
    for (int64_t j = symmetric ? i : 0; j < ms; ++j) cnt[rank.at(kq[i] + ks[j]) + 1]++;
  out.ptr.assign(mo + 1, 0);
  for (int64_t k = 0; k < mo; ++k) out.ptr[k + 1] = out.ptr[k] + cnt[k + 1];
  out.pairs.assign((size_t)out.ptr[mo], 0);
  std::vector<int32_t> fill(out.ptr.begin(), out.ptr.end() - 1);
  for (int64_t i = 0; i < mq; ++i)
    for (int64_t j = symmetric ? i : 0; j < ms; ++j) {
      int32_t k = rank.at(kq[i] + ks[j]);
      out.pairs[(size_t)fill[k]++] = (uint32_t)i | ((uint32_t)j << 16);
    }
  out.m_in = mq;
  out.m_out = mo;
  return true;
}

bool build_square_pairs(int n, int D, PairList& out) {
  return build_pairs(n, D, D, true, out);
}

bool build_product_table(int n, int Dq, int Ds, int64_t max_pairs, std::vector<int32_t>& ptr,
                         std::vector<int32_t>& pairs) {
  const int64_t mq = num_monomials(n, Dq), ms = num_monomials(n, Ds);
  const int64_t mo = num_monomials(n, Dq + Ds);
  if (mq < 0 || ms < 0 || mo < 0 || mq * ms > max_pairs || mo > INT32_MAX - 1) return false;
  std::vector<uint8_t> ex;
  graded_monomials(n, Dq + Ds, ex);
  std::unordered_map<uint64_t, int32_t> rank;
  rank.reserve((size_t)mo * 2);
  for (int64_t r = 0; r < mo; ++r) rank[pack_key(&ex[(size_t)r * n], n)] = (int32_t)r;
  // the graded order of degree <= D is a prefix of the list, so the ranks of
  // q's and s's monomials are their ranks in ex
  std::vector<int32_t> code((size_t)mq * ms);
  std::vector<int32_t> cnt(mo + 1, 0);
  for (int64_t i = 0; i < mq; ++i) {
    const uint64_t ki = pack_key(&ex[(size_t)i * n], n);
    for (int64_t j = 0; j < ms; ++j) {
      const int32_t k = rank.at(ki + pack_key(&ex[(size_t)j * n], n));
      code[(size_t)i * ms + j] = k;
      cnt[k + 1]++;
    }
  }
  ptr.assign(mo + 1, 0);
  for (int64_t k = 0; k < mo; ++k) ptr[k + 1] = ptr[k] + cnt[k + 1];
  pairs.assign((size_t)ptr[mo] * 2, 0);
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < mq; ++i)
    for (int64_t j = 0; j < ms; ++j) {
      const int32_t p = fill[code[(size_t)i * ms + j]]++;
      pairs[(size_t)p * 2] = (int32_t)i;
      pairs[(size_t)p * 2 + 1] = (int32_t)j;
    }
  return true;
}

bool build_row_table(int n, int D, RowImage& out) {
  out = RowImage{};
  if (D < 0 || D > kMaxRowDegree) return false;
  const int64_t m_in = num_monomials(n, D);
  const int64_t m_full = num_monomials(n, 2 * D);
  // prefixes: exponent vectors of t_1..t_{n-1} up to total degree 2D
  std::vector<uint8_t> pre;
  int np;
  if (n == 1) {
    np = 1;
  } else {
    graded_monomials(n - 1, 2 * D, pre);
    np = (int)num_monomials(n - 1, 2 * D);
  }
  auto psum = [&](int i) {
    int s = 0;
    for (int k = 0; k < n - 1; ++k) s += pre[(size_t)i * (n - 1) + k];
    return s;
  };
  std::vector<uint8_t> ex;
  graded_monomials(n, 2 * D, ex);
  std::unordered_map<uint64_t, int32_t> rank;
  rank.reserve((size_t)m_full * 2);
  for (int64_t r = 0; r < m_full; ++r) rank[pack_key(&ex[(size_t)r * n], n)] = (int32_t)r;
  auto full_rank = [&](int pi, int c) {
    uint8_t e[kMaxVars] = {0};
    for (int k = 0; k < n - 1; ++k) e[k] = pre[(size_t)pi * (n - 1) + k];
    e[n - 1] = (uint8_t)c;
    return rank.at(pack_key(e, n));
  };
  // input rows: the prefixes of degree <= D (a graded prefix of the list)
  const int np_in = n == 1 ? 1 : (int)num_monomials(n - 1, D);
  std::vector<int32_t> off(np_in), len(np_in);
  int pos = 0;
  out.pos_in.assign(m_in, -1);
  for (int i = 0; i < np_in; ++i) {
    off[i] = pos;
    len[i] = D - (n == 1 ? 0 : psum(i)) + 1;
    for (int c = 0; c < len[i]; ++c) out.pos_in[full_rank(i, c)] = pos + c;
    pos += len[i];
  }
  if (pos != m_in) return false;
  // prefix key -> prefix index
  std::unordered_map<uint64_t, int32_t> pidx;
  for (int i = 0; i < np; ++i) pidx[n == 1 ? 0 : pack_key(&pre[(size_t)i * (n - 1)], n - 1)] = i;
  std::vector<std::vector<int>> bucket(np);
  for (int i = 0; i < np_in; ++i)
    for (int j = i; j < np_in; ++j) {
      uint64_t k = 0;
      if (n > 1)
        k = pack_key(&pre[(size_t)i * (n - 1)], n - 1) + pack_key(&pre[(size_t)j * (n - 1)], n - 1);
      bucket[pidx.at(k)].push_back(i * np_in + j);
    }
  out.n_out_rows = np;
  out.m_in = (int)m_in;
  for (int P = 0; P < np; ++P) {
    const int sP = n == 1 ? 0 : psum(P);
    const int Lout = 2 * D - sP + 1;
    out.hdr.push_back((int32_t)(out.pairs.size() / 4));
    // off-diagonal pairs first, then the diagonal pair (p == q) if P = 2p
    int has_diag = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int code : bucket[P]) {
        const int i = code / np_in, j = code % np_in;
        if ((i == j) != (pass == 1)) continue;
        has_diag |= (i == j);
        int oi = off[i], oj = off[j], li = len[i], lj = len[j];
        if (li > lj) {
          std::swap(oi, oj);
          std::swap(li, lj);
        }
        out.pairs.push_back(oi);
        out.pairs.push_back(oj);
        out.pairs.push_back((li << 4) | lj);
        out.pairs.push_back(row_pair_case(li, lj));
      }
    out.hdr.push_back((int32_t)(out.pairs.size() / 4));
    out.hdr.push_back((int32_t)out.out_ranks.size());
    const int in_len = sP <= D ? D - sP + 1 : 0;
    out.hdr.push_back(Lout | (in_len << 8) | (has_diag << 16));
    out.in_off.push_back(sP <= D ? off[P] : -1);
    for (int c = 0; c < Lout; ++c) out.out_ranks.push_back(full_rank(P, c));
  }
  // split the output rows into two ranges of about equal work (products of
  // row lengths plus a cost per output element)
  std::vector<int64_t> work(np, 0);
  for (int P = 0; P < np; ++P) {
    for (int k = out.hdr[4 * P]; k < out.hdr[4 * P + 1]; ++k) {
      const int code = out.pairs[4 * k + 2];
      work[P] += (int64_t)(code >> 4) * (code & 15) + 6;
    }
    work[P] += 8 * (out.hdr[4 * P + 3] & 0xff);
  }
  int64_t total = 0;
  for (int64_t w : work) total += w;
  int64_t run = 0;
  out.row_split = np;
  for (int P = 0; P < np; ++P) {
    if (2 * run >= total) {
      out.row_split = P;
      break;
    }
    run += work[P];
  }
  if (out.row_split == 0) out.row_split = std::min(1, np);
  return true;
}

// The row-convolution kernel keeps one row-layout copy of the input per lane
// in shared memory (32 lanes per warp); inputs up to 750 terms fit one warp in
// 96 KB.
int row_path_max_degree(int n) {
  int D = kMaxRowDegree;
  while (D > 0 && num_monomials(n, D) > 750) --D;
  return D;
}

void build_degree_of(int n, int De, std::vector<uint8_t>& out) {
  const int64_t m = num_monomials(n, De);
  out.assign((size_t)m + 1, 0);
  int D = 0;
  for (int64_t c = 0; c <= m; ++c) {
    while (num_monomials(n, D) < c) ++D;
    out[(size_t)c] = (uint8_t)D;
  }
}

int max_enclose_order(int n) {
  int l = kMaxEncloseOrder;
  for (; l > 0; --l) {
    int64_t g = 1;
    for (int k = 0; k < n; ++k) g *= (l + 1);
    if (g <= BERN_MAX_GRID) break;
  }
  return l;
}

int max_enclose_order_big(int n) {
  int l = kMaxEncloseOrder;
  for (; l > 0; --l) {
    int64_t g = 1;
    for (int k = 0; k < n && g <= BERN_MAX_BIG_GRID; ++k) g *= (l + 1);
    if (g <= BERN_MAX_GRID || (g <= BERN_MAX_BIG_GRID && l <= 16)) break;
  }
  return std::max(l, max_enclose_order(n));
}

void build_rscale(int n, int l, std::vector<float>& out) {
  std::vector<uint8_t> ex;
  graded_monomials(n, l, ex);
  const int64_t m = num_monomials(n, l);
  out.assign((size_t)m * 2, 0.0f);
  for (int64_t r = 0; r < m; ++r) {
    unsigned __int128 c = 1;
    for (int k = 0; k < n; ++k) {
      const int e = ex[(size_t)r * n + k];
      unsigned long long b = 1;
      for (int i = 1; i <= e; ++i) b = b * (unsigned long long)(l - e + i) / (unsigned long long)i;
      c *= b;
    }
    float lo, hi;
    if ((c & (c - 1)) == 0) {             // a power of two: the reciprocal is exact
      lo = hi = (float)(1.0L / (long double)c);
    } else {
      const float f = (float)(1.0L / (long double)c);
      lo = std::nextafter(f, 0.0f);       // |f - 1/c| < 1 ulp, so lo < 1/c < hi
      hi = std::nextafter(f, 1.0f);
    }
    out[(size_t)r * 2] = lo;
    out[(size_t)r * 2 + 1] = hi;
  }
}

}  // namespace bern

namespace bern {

// Enclosure index tables for order l (grid radix R = l + 1, variable 0 the
// slowest digit): gidx[r] = grid index of graded rank r < M(n, l); lines
// holds, for each variable k and each line Ln along k (Ln enumerates the
// digits of the other variables, the highest variable first), the pair
// (base offset, digit sum of the variables before k).
void build_enclose_tables(int n, int l, std::vector<int32_t>& gidx, std::vector<int32_t>& lines,
                          bool with_lines) {
  const int R = l + 1;
  std::vector<int64_t> pw(n);
  int64_t p = 1;
  for (int k = n - 1; k >= 0; --k) {
    pw[k] = p;
    p *= R;
  }
  std::vector<uint8_t> ex;
  graded_monomials(n, l, ex);
  const int64_t m = num_monomials(n, l);
  gidx.assign((size_t)m, 0);
  for (int64_t r = 0; r < m; ++r) {
    int64_t ix = 0;
    for (int k = 0; k < n; ++k) ix += ex[(size_t)r * n + k] * pw[k];
    gidx[(size_t)r] = (int32_t)ix;
  }
  lines.clear();
  if (!with_lines) return;
  int64_t nlines = 1;
  for (int k = 0; k < n - 1; ++k) nlines *= R;
  lines.assign((size_t)(2 * n * nlines), 0);
  for (int k = 0; k < n; ++k)
    for (int64_t Ln = 0; Ln < nlines; ++Ln) {
      int64_t rest = Ln, base = 0;
      int psum = 0;
      for (int mm = n - 1; mm >= 0; --mm) {
        if (mm == k) continue;
        const int dgt = (int)(rest % R);
        rest /= R;
        base += dgt * pw[mm];
        if (mm < k) psum += dgt;
      }
      lines[(size_t)(2 * (k * nlines + Ln))] = (int32_t)base;
      lines[(size_t)(2 * (k * nlines + Ln)) + 1] = psum;
    }
  // within a pass the lines are independent: from four variables on (where
  // the simplex is a small part of the grid) the lines whose prefix digit
  // sum is <= l (all a polynomial of degree <= l can need) come first, the
  // first C(l + k, k) * (l+1)^(n-1-k) of pass k, each group in its natural
  // order (neighbouring lanes keep neighbouring grid offsets)
  if (n < 4) return;
  std::vector<std::pair<int32_t, int32_t>> tmp((size_t)nlines);
  for (int k = 0; k < n; ++k) {
    int32_t* pl = &lines[(size_t)(2 * k * nlines)];
    for (int64_t Ln = 0; Ln < nlines; ++Ln) tmp[(size_t)Ln] = {pl[2 * Ln + 1], pl[2 * Ln]};
    std::stable_partition(tmp.begin(), tmp.end(),
                          [l](const std::pair<int32_t, int32_t>& a) { return a.first <= l; });
    for (int64_t Ln = 0; Ln < nlines; ++Ln) {
      pl[2 * Ln] = tmp[(size_t)Ln].second;
      pl[2 * Ln + 1] = tmp[(size_t)Ln].first;
    }
  }
}

}  // namespace bern

namespace bern {

int device_sms(const Launch& L) {
  if (L.sms > 0) return L.sms;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return 1;
  return sms;
}

int tune_variant(const Launch& L, const char* kind, const std::string& key, int dflt) {
  if (!L.tuner) return dflt;
  if (!L.tuner->probe_kind.empty())
    return L.tuner->probe_kind == kind ? L.tuner->probe_variant : dflt;
  auto f = L.tuner->forced.find(kind);
  if (f != L.tuner->forced.end()) return f->second;
  auto it = L.tuner->best.find(key);
  return it == L.tuner->best.end() ? dflt : it->second;
}

void tune_begin(const Launch& L, const char* kind, TuneTimer& t) {
  t.on = L.tuner && L.tuner->probe_kind == kind;
  if (!t.on) return;
  cudaEventCreate(&t.e0);
  cudaEventCreate(&t.e1);
  cudaEventRecord(t.e0, L.stream);
}

void tune_end(const Launch& L, const char* kind, const std::string& key, TuneTimer& t) {
  if (!t.on) return;
  cudaEventRecord(t.e1, L.stream);
  cudaEventSynchronize(t.e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, t.e0, t.e1);
  cudaEventDestroy(t.e0);
  cudaEventDestroy(t.e1);
  auto& v = L.tuner->probe_ms[key];
  const int var = L.tuner->probe_variant;
  if ((int)v.size() <= var) v.resize(var + 1, -1.0f);
  v[var] = (v[var] < 0.0f ? 0.0f : v[var]) + ms;
  (void)kind;
}

}  // namespace bern
