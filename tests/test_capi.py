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


def test_binding_return_types_follow_the_header(lib):
    """Each function's ctypes return type matches its declaration (a 64-bit
    count read as a C int would wrap above 2^31)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"^\s*((?:const\s+)?[a-z_0-9]+\s*\**)\s*(rbf_[a-z_0-9]+)\s*\(", text, flags=re.M)
    want = {"rbf_status": C.c_int, "int": C.c_int, "int64_t": C.c_int64, "uint64_t": C.c_uint64,
            "double": C.c_double, "void": None, "constchar*": C.c_char_p}
    seen = 0
    for ret, name in decls:
        key = re.sub(r"\s+", "", ret)
        assert key in want, (name, ret)
        got = getattr(lib, name).restype
        exp = want[key]
        if exp is None:
            assert got is None, name
        else:
            assert got is not None and C.sizeof(got) == C.sizeof(exp), (name, got, exp)
            assert (got in (C.c_char_p, C.c_double)) == (exp in (C.c_char_p, C.c_double)), name
        seen += 1
    assert seen == len(header_functions())


def test_binding_constants_follow_the_header():
    """Options, profiler classes, precisions and status codes: the values the
    binding passes are the header's."""
    from paper_0909_5413_gb300 import rbf
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {name: int(val) for name, val in re.findall(r"\b(RBF_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    assert len(consts) >= 28
    for name, val in consts.items():
        if name.startswith(("RBF_OPT_", "RBF_PROF_", "RBF_FP")):
            assert getattr(rbf, name) == val, name
        else:   # status codes
            assert rbf.STATUS_NAMES[val] == name, name
    assert len(rbf.STATUS_NAMES) == sum(1 for n in consts if not n.startswith(("RBF_OPT_", "RBF_PROF_", "RBF_FP")))


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


def test_server_rejects_bad_parameters_without_gpu(lib):
    from paper_0909_5413_gb300 import rbf
    h = C.c_void_p()
    for slots in (0, 65):
        p = rbf.RbfServerParams(0, slots, 0)
        assert lib.rbf_server_create(C.byref(h), C.byref(p)) == 1
    p = rbf.RbfServerParams(0, 2, -5)
    assert lib.rbf_server_create(C.byref(h), C.byref(p)) == 1
    assert lib.rbf_server_submit(None, None, None) == 1
    assert lib.rbf_server_clock(None) == 0.0


def test_request_footprint_estimate(lib):
    """The admission estimate (host only): grows in proportion to N, and the
    mixed form with FP32 inverses needs about half the bytes of the FP64 form."""
    import numpy as np
    from paper_0909_5413_gb300 import rbf
    from paper_0909_5413_gb300 import workloads as W

    def fp(n_side, mixed):
        p = W.lattice_problem(n_side, 0.8, seed=1)
        cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64)
        w = np.zeros(p.n)
        return rbf.rbf_request_footprint(rbf.make_request(p.xy, p.f, w, cfg)), p.n

    f64_small, n_small = fp(64, False)
    f64_big, n_big = fp(256, False)
    mix_big, _ = fp(256, True)
    fixed = 16 << 20
    per_small = (f64_small - fixed) / n_small
    per_big = (f64_big - fixed) / n_big
    assert abs(per_small - per_big) / per_big < 0.05
    # FP64: staging, lists, 31 Krylov vectors (248 B) and 36 FP64 inverse entries per point (288 B)
    assert 600 < per_big < 800
    assert 0.4 < (mix_big - fixed) / (f64_big - fixed) < 0.65
    assert rbf.rbf_request_footprint(rbf.RbfRequest()) == 0
