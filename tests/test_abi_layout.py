"""The Python binding's ctypes structs match include/bern.h byte for byte:
a small C program compiled here with the host compiler prints the size and
every field offset of the header's structs, and the binding's ctypes
definitions must give the same numbers.  No GPU and no library call."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2211_14438_gb300 import bern

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "bern_net": (bern.bern_net, ["n_layers", "widths", "W", "b"]),
    "bern_mlp": (bern.bern_mlp, ["n_features", "n_classes", "W1", "b1", "W2", "b2"]),
    "bern_degree_plan": (bern.bern_degree_plan,
                         ["kind", "global_d", "per_layer", "per_neuron", "degree_cap",
                          "prune_tau", "bern_budget", "mlp", "min_conf", "lin_every"]),
    "bern_result": (bern.bern_result, ["lo", "hi", "n_terms", "keys", "coef", "cap_terms"]),
    "bern_trace": (bern.bern_trace, ["lo", "hi", "nterms", "degree"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bern.h"', "int main(void) {"]
    for name, (_, fields) in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f in fields:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_matches_header(c_layout, name):
    cls, fields = STRUCTS[name]
    assert ctypes.sizeof(cls) == c_layout[(name, "size")], name
    assert [f[0] for f in cls._fields_] == fields
    for f in fields:
        assert getattr(cls, f).offset == c_layout[(name, f)], (name, f)


def _header_prototypes():
    import re
    src = open(os.path.join(ROOT, "include", "bern.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(bern_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src):
        ret, name, params = m.group(1), m.group(2), m.group(3)
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        protos[name] = (ret.strip(), ps)
    return protos


def _kind_of_c(decl):
    if "*" in decl:
        return "ptr"
    t = decl.replace("const", "").split()[0]
    return {"int": "i32", "int64_t": "i64", "float": "f32", "double": "f64"}[t]


def _kind_of_ctypes(t):
    if t in (ctypes.c_int, ctypes.c_int32):
        return "i32"
    if t in (ctypes.c_int64, ctypes.c_longlong):
        return "i64"
    if t is ctypes.c_float:
        return "f32"
    if t is ctypes.c_double:
        return "f64"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    raise AssertionError(t)


def test_function_signatures_match_header():
    lib = bern.load()
    protos = _header_prototypes()
    assert set(protos) == set(bern.EXPORTS)
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        got = [_kind_of_ctypes(t) for t in fn.argtypes]
        want = [_kind_of_c(p) for p in params]
        assert got == want, (name, got, want)
        assert _kind_of_ctypes(fn.restype) == _kind_of_c(ret + (" *" if "*" in ret else "")), name
