"""C-ABI library checks that need no GPU: it builds, loads, and exports every
function include/rbf.h declares; the Python binding names the same set."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbf.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rbf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_0909_5413_gb300 import build
    build.build()
    from paper_0909_5413_gb300 import rbf
    return rbf.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("rbf_bin", "rbf_matvec", "rbf_rasm_setup", "rbf_rasm_apply", "rbf_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    from paper_0909_5413_gb300 import rbf
    assert sorted(rbf.EXPORTED) == header_functions()


def test_status_strings(lib):
    from paper_0909_5413_gb300 import rbf
    assert rbf.rbf_status_string(0) == "ok"
    assert "converged" in rbf.rbf_status_string(6)
    assert rbf.rbf_status_string(99) == "unknown status"


def test_null_context_is_rejected_without_gpu(lib):
    from paper_0909_5413_gb300 import rbf
    p = rbf.RbfParams(1.0, 8.6, 0.0, 0)
    assert lib.rbf_bin(None, None, 10, C.byref(p), None) == 1
    assert lib.rbf_launch_count(None) == 0
    assert lib.rbf_last_error(None) == b"null context"
