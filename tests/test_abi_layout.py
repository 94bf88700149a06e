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
