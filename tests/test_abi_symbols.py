"""The C-ABI library builds, loads without a GPU and exports every function include/hisq.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "hisq.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(hisq_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1409_1510_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared()
    for required in ("hisq_dslash", "hisq_cg_solve", "hisq_init", "hisq_links_create", "hisq_aop",
                     "hisq_pc_apply", "hisq_pc_train"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_calls_without_context_fail_cleanly(lib):
    from paper_1409_1510_gb300 import hisq
    hisq.load()
    assert lib.hisq_finalize() == -7
    assert hisq.hisq_strerror(-4).startswith("solver did not converge")


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program compiled against include/hisq.h."""
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hisq.h"', "int main(void) {",
             f'    printf("%zu\\n", sizeof({struct}));']
    lines += [f'    printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["hisq_solver_params", "hisq_solve_stats"])
def test_binding_structs_match_the_header(name, tmp_path):
    """The ctypes mirrors of the parameter and statistics structs have the header's layout."""
    from paper_1409_1510_gb300 import hisq
    cls = getattr(hisq, name)
    fields = [f for f, _ in cls._fields_]
    size, offsets = _c_layout(name, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets
