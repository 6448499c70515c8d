"""The C-ABI library builds, loads without a GPU and exports every function include/hisq.h declares."""
import ctypes
import os
import re

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
