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
