"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/bern.h declares, and its host-side
monomial tables are right.  No compute call touches a GPU here."""
import ctypes
import itertools
import math
import os
import re

import numpy as np
import pytest

from paper_2211_14438_gb300 import bern

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bern.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bern_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    names = declared_functions()
    assert len(names) >= 14
    assert set(names) == set(bern.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(bern.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_codes():
    for code in range(8):
        assert bern.strerror(code)
    assert bern.strerror(0) == "ok"
    assert bern.strerror(99) == "unknown status"


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_num_monomials_matches_binomial(n):
    for D in (0, 1, 2, 5, 8, 16):
        assert bern.num_monomials(n, D) == math.comb(n + D, n)
    assert bern.num_monomials(0, 3) == -1 and bern.num_monomials(9, 3) == -1
    assert bern.num_monomials(n, 65) == -1


@pytest.mark.parametrize("n,D", [(1, 6), (2, 5), (3, 4), (4, 3), (6, 2)])
def test_graded_order(n, D):
    ex = bern.monomials(n, D).astype(int)
    every = {e for e in itertools.product(range(D + 1), repeat=n) if sum(e) <= D}
    assert len(ex) == len(every) and {tuple(r) for r in ex} == every
    deg = ex.sum(1)
    assert np.all(np.diff(deg) >= 0)                     # graded: prefix property
    for g in range(D + 1):                               # descending lex within a degree
        block = [tuple(r) for r in ex[deg == g]]
        assert block == sorted(block, reverse=True)
        assert bern.num_monomials(n, g) == int((deg <= g).sum())
    # degree-1 block is t_1, ..., t_n in order
    assert [tuple(r) for r in ex[1:n + 1]] == [tuple(np.eye(n, dtype=int)[i]) for i in range(n)]


# ------------------------------------------------------------ enclosure line tables
def _digits(idx, n, R):
    """Digits (d_0 .. d_{n-1}) of a grid index, variable 0 the slowest."""
    d = []
    for _ in range(n):
        d.append(idx % R)
        idx //= R
    return d[::-1]


def _natural_index(d, k, R):
    """A line's place in the natural order: the digits of the variables other
    than k read as one number whose lowest digit is the highest variable."""
    idx, w = 0, 1
    for mm in range(len(d) - 1, -1, -1):
        if mm == k:
            continue
        idx += d[mm] * w
        w *= R
    return idx


@pytest.mark.parametrize("n,l", [(1, 5), (2, 4), (3, 0), (3, 4), (3, 8), (3, 16), (4, 3),
                                 (4, 6), (5, 3), (6, 2), (6, 4), (8, 2)])
def test_enclose_lines_cover_every_line_once(n, l):
    # Def. 2's per-variable transform runs along every line of the grid once:
    # pass k holds each cell with d_k = 0 once, with the digit sum of the
    # variables before k
    R = l + 1
    t = bern.enclose_lines(n, l)
    assert t.shape == (n, R ** (n - 1), 2)
    for k in range(n):
        bases = t[k, :, 0].tolist()
        want = {i for i in range(R ** n) if _digits(i, n, R)[k] == 0}
        assert len(bases) == len(want) and set(bases) == want
        for base, psum in t[k].tolist():
            assert psum == sum(_digits(base, n, R)[:k])


@pytest.mark.parametrize("l", [0, 1, 2, 4, 7, 8, 11, 16])
def test_enclose_lines_three_variables_match_the_kernel_formulas(l):
    # the three-variable enclosure kernels compute a line's entries from its
    # index Ln instead of loading them; they must equal the table's
    R = l + 1
    t = bern.enclose_lines(3, l)
    for Ln in range(R * R):
        q, r = divmod(Ln, R)
        assert tuple(t[2, Ln]) == (Ln * R, q + r)
        assert tuple(t[1, Ln]) == (q * R * R + r, q)
        assert tuple(t[0, Ln]) == (Ln, 0)


@pytest.mark.parametrize("n,l", [(1, 6), (2, 5), (3, 6), (4, 2), (4, 5), (5, 3), (6, 2),
                                 (6, 4), (7, 2), (8, 2)])
def test_enclose_lines_order(n, l):
    # below four variables: natural order; from four on, the lines of prefix
    # sum <= l (C(l+k, k) (l+1)^(n-1-k) of them, the loop bound of the
    # kernels there) first, then the rest, each part in natural order
    R = l + 1
    t = bern.enclose_lines(n, l)
    for k in range(n):
        nat = [_natural_index(_digits(b, n, R), k, R) for b in t[k, :, 0].tolist()]
        psum = t[k, :, 1]
        if n < 4:
            assert nat == list(range(R ** (n - 1)))
            continue
        cnt = math.comb(l + k, k) * R ** (n - 1 - k)
        assert np.all(psum[:cnt] <= l) and np.all(psum[cnt:] > l)
        assert nat[:cnt] == sorted(nat[:cnt]) and nat[cnt:] == sorted(nat[cnt:])


def test_enclose_lines_rejects_bad_arguments():
    lib = bern.load()
    buf = np.zeros(64, np.int32)
    assert lib.bern_enclose_lines(3, 2, None, 64) == 1             # BERN_E_INVALID
    assert lib.bern_enclose_lines(0, 2, buf.ctypes.data, 64) == 1
    assert lib.bern_enclose_lines(9, 2, buf.ctypes.data, 64) == 1
    assert lib.bern_enclose_lines(3, -1, buf.ctypes.data, 64) == 1
    assert lib.bern_enclose_lines(3, 4, buf.ctypes.data, 64) == 1   # needs 2*3*25 = 150
    assert lib.bern_enclose_lines(3, 2, buf.ctypes.data, 64) == 0   # 2*3*9 = 54 fit
    assert lib.bern_enclose_lines(2, (1 << 11) + 1, buf.ctypes.data, 64) == 6   # > 2^22 cells


@pytest.mark.parametrize("n,l", [(1, 0), (1, 16), (1, 24), (2, 8), (3, 4), (3, 8), (3, 16),
                                 (4, 6), (6, 4), (8, 2)])
def test_enclose_scales_bracket_the_reciprocals(n, l):
    # Def. 2 divides a_J by prod_k C(l, j_k); the kernels multiply by a float
    # bracket of the reciprocal, so each pair must contain it exactly and be
    # tight (one float when the product is a power of two, else two ulps wide)
    from fractions import Fraction
    sc = bern.enclose_scales(n, l).astype(np.float64)
    ex = bern.monomials(n, l).astype(int)
    assert sc.shape == (len(ex), 2)
    for (lo, hi), J in zip(sc, ex):
        c = 1
        for j in J:
            c *= math.comb(l, int(j))
        exact = Fraction(1, c)
        assert Fraction(lo) <= exact <= Fraction(hi)
        if c & (c - 1) == 0:
            assert lo == hi == float(exact)
        else:
            assert Fraction(lo) < exact < Fraction(hi)
            one = np.float32(1)
            assert np.nextafter(np.nextafter(np.float32(lo), one), one) == np.float32(hi)


def test_enclose_scales_rejects_bad_arguments():
    lib = bern.load()
    buf = np.zeros(64, np.float32)
    assert lib.bern_enclose_scales(3, 2, None, 64) == 1
    assert lib.bern_enclose_scales(0, 2, buf.ctypes.data, 64) == 1
    assert lib.bern_enclose_scales(3, 25, buf.ctypes.data, 64) == 1
    assert lib.bern_enclose_scales(3, 4, buf.ctypes.data, 64) == 1    # needs 2 * 35 = 70
    assert lib.bern_enclose_scales(3, 2, buf.ctypes.data, 64) == 0    # 2 * 10 = 20 fit


# ------------------------------------------------------------ composition row tables
_CASES = {}


@pytest.mark.parametrize("n,D", [(1, 0), (1, 8), (2, 3), (2, 8), (3, 0), (3, 1), (3, 2), (3, 4),
                                 (3, 8), (4, 5), (5, 4), (6, 3), (8, 2)])
def test_compose_rows_give_the_exact_square(n, D):
    # Step 3 at ReLU order 2 forms a1 s + a2 s^2; replay the row kernel's
    # reading of the tables (off-diagonal row pairs counted twice, the
    # diagonal pair as a triangle, the row's own input row as the linear
    # term, each output element to its graded rank) on integer coefficients
    # and compare with the product expanded monomial by monomial
    t = bern.compose_rows(n, D)
    ex_in = bern.monomials(n, D).astype(int)
    ex_out = bern.monomials(n, 2 * D).astype(int)
    rank_out = {tuple(e): r for r, e in enumerate(ex_out)}
    M = len(ex_in)
    rng = np.random.default_rng(31 * n + D)
    p = rng.integers(-9, 10, M).astype(np.int64)
    a1, a2 = 3, 5
    want = np.zeros(len(ex_out), np.int64)
    for i in range(M):
        want[rank_out[tuple(ex_in[i])]] += a1 * p[i]
        for j in range(M):
            want[rank_out[tuple(ex_in[i] + ex_in[j])]] += a2 * p[i] * p[j]

    assert sorted(t["pos_in"].tolist()) == list(range(M))
    s = np.zeros(M, np.int64)
    s[t["pos_in"]] = p
    unset = np.iinfo(np.int64).min
    got = np.full(len(ex_out), unset, np.int64)
    for P, (pb, pe, rb, w) in enumerate(t["hdr"].tolist()):
        Lout, in_len, has_diag = w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 1
        acc = np.zeros(Lout, np.int64)
        for k in range(pb, pe - has_diag):
            op, oq, code, case = t["pairs"][k].tolist()
            L1, L2 = code >> 4, code & 15
            assert 1 <= L1 <= L2 <= 9 and op + L1 <= M and oq + L2 <= M
            assert _CASES.setdefault((L1, L2), case) == case
            for a in range(L1):
                for b in range(L2):
                    acc[a + b] += 2 * s[op + a] * s[oq + b]
        if has_diag:
            o, _, code, case = t["pairs"][pe - 1].tolist()
            L = code & 15
            assert code >> 4 == L and o + L <= M
            assert _CASES.setdefault((L, L), case) == case
            for a in range(L):
                acc[2 * a] += s[o + a] * s[o + a]
                for b in range(a + 1, L):
                    acc[a + b] += 2 * s[o + a] * s[o + b]
        for c in range(Lout):
            lin = s[t["in_off"][P] + c] if c < in_len else 0
            r = t["out_ranks"][rb + c]
            assert got[r] == unset                       # every rank written once
            got[r] = a2 * acc[c] + a1 * lin
    assert np.array_equal(got, want)
    assert 0 <= t["row_split"] <= len(t["hdr"])
    # the dispatch cases seen so far: one per pair of row lengths, all distinct
    # and inside the dense range of the kernel's switch
    assert len(set(_CASES.values())) == len(_CASES)
    assert all(0 <= v < 45 for v in _CASES.values())


def test_compose_rows_limits():
    lib = bern.load()
    sizes = np.zeros(5, np.int64)
    assert lib.bern_compose_rows(3, 8, None, 0, None) == 1          # sizes NULL
    assert lib.bern_compose_rows(3, 9, None, 0, sizes.ctypes.data) == 1
    assert lib.bern_compose_rows(6, 8, None, 0, sizes.ctypes.data) == 6   # 3003 terms
    assert lib.bern_compose_rows(3, 8, None, 0, sizes.ctypes.data) == 0
    assert sizes[0] == math.comb(11, 3)
    buf = np.zeros(8, np.int32)
    assert lib.bern_compose_rows(3, 8, buf.ctypes.data, buf.size, sizes.ctypes.data) == 1


# ------------------------------------------------------------ composition pair lists
@pytest.mark.parametrize("n,Dq,Ds,square", [
    (1, 4, 4, True), (2, 3, 3, True), (3, 4, 4, True), (3, 8, 8, True), (6, 2, 2, True),
    (1, 3, 5, False), (2, 4, 2, False), (3, 8, 2, False), (3, 16, 2, False), (6, 4, 2, False)])
def test_pair_lists_give_the_exact_product(n, Dq, Ds, square):
    # every pair of output K's list has I + J = K, every pair of input
    # monomials (I <= J for the square) appears once, and the products read
    # off the lists (the square's off-diagonal pairs counted twice) are exact
    ptr, pairs = bern.pair_lists(n, Dq, Ds, square)
    ex = bern.monomials(n, Dq + Ds).astype(int)
    mq, ms, mo = (bern.num_monomials(n, D) for D in (Dq, Ds, Dq + Ds))
    assert len(ptr) == mo + 1 and ptr[0] == 0 and ptr[-1] == len(pairs)
    assert np.all(np.diff(ptr) >= 0)
    seen = set()
    for K in range(mo):
        for I, J in pairs[ptr[K]:ptr[K + 1]].tolist():
            assert I < mq and J < ms and np.array_equal(ex[I] + ex[J], ex[K])
            assert (I <= J) or not square
            assert (I, J) not in seen
            seen.add((I, J))
    assert len(seen) == (mq * (mq + 1) // 2 if square else mq * ms)

    rng = np.random.default_rng(7 * n + Dq + 3 * Ds)
    q = rng.integers(-9, 10, mq).astype(np.int64)
    s = q if square else rng.integers(-9, 10, ms).astype(np.int64)
    rank = {tuple(e): r for r, e in enumerate(ex)}
    want = np.zeros(mo, np.int64)
    for i in range(mq):
        for j in range(ms):
            want[rank[tuple(ex[i] + ex[j])]] += q[i] * s[j]
    got = np.zeros(mo, np.int64)
    for K in range(mo):
        for I, J in pairs[ptr[K]:ptr[K + 1]].tolist():
            got[K] += q[I] * s[J] * (2 if square and I != J else 1)
    assert np.array_equal(got, want)


def test_pair_lists_limits():
    lib = bern.load()
    sizes = np.zeros(2, np.int64)
    assert lib.bern_pair_lists(3, 2, 2, 1, None, 0, None, 0, None) == 1
    assert lib.bern_pair_lists(3, 2, 3, 1, None, 0, None, 0, sizes.ctypes.data) == 1   # square, Dq != Ds
    assert lib.bern_pair_lists(9, 2, 2, 1, None, 0, None, 0, sizes.ctypes.data) == 1
    assert lib.bern_pair_lists(3, 40, 30, 0, None, 0, None, 0, sizes.ctypes.data) == 1  # degree > 64
    assert lib.bern_pair_lists(3, 2, 2, 1, None, 0, None, 0, sizes.ctypes.data) == 0
    assert sizes.tolist() == [math.comb(7, 3) + 1, 10 * 11 // 2]
    assert lib.bern_pair_lists(4, 16, 16, 0, None, 0, None, 0, sizes.ctypes.data) == 6   # > 2^24 pairs
    p = np.zeros(4, np.int32)
    assert lib.bern_pair_lists(3, 2, 2, 1, p.ctypes.data, 4, p.ctypes.data, 4,
                               sizes.ctypes.data) == 1                              # caps too small
