"""Thin ctypes binding of ``librbf.so`` (include/rbf.h).

Functions carry the C names and only marshal arguments: torch tensors are
passed as raw device pointers, streams as ``cudaStream_t`` handles. Every step
of the computation runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback, and a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbf.so")

RBF_FP64 = 0
RBF_FP32 = 1
RBF_FP32_FROM_FP64 = 2

STATUS_NAMES = {0: "RBF_OK", 1: "RBF_ERR_INVALID_ARG", 2: "RBF_ERR_OOM", 3: "RBF_ERR_CUDA", 4: "RBF_ERR_NOT_SPD",
                5: "RBF_ERR_SUBDOMAIN_TOO_LARGE", 6: "RBF_ERR_NOT_CONVERGED", 7: "RBF_ERR_TIMEOUT",
                8: "RBF_ERR_STATE"}

# Every function include/rbf.h declares.
EXPORTED = ["rbf_create", "rbf_destroy", "rbf_bin", "rbf_matvec", "rbf_rasm_setup", "rbf_rasm_apply", "rbf_solve",
            "rbf_interpolate_host", "rbf_get_grid", "rbf_get_bins", "rbf_get_subdomain_sizes", "rbf_get_subdomains",
            "rbf_count_neighbors", "rbf_get_neighbors", "rbf_status_string", "rbf_last_error", "rbf_launch_count",
            "rbf_device_bytes", "rbf_profile_enable", "rbf_profile_read", "rbf_debug_exp", "rbf_matvec_noalloc",
            "rbf_bin_batch", "rbf_rasm_setup_batch", "rbf_solve_batch", "rbf_server_create", "rbf_server_destroy",
            "rbf_server_submit", "rbf_server_wait", "rbf_server_get_stats", "rbf_server_clock",
            "rbf_request_footprint", "rbf_debug_kernel_pairs", "rbf_eval", "rbf_tune",
            "rbf_count_candidates", "rbf_profile_classes", "rbf_set_memory_limit",
            "rbf_count_pairs", "rbf_rasm_factor_counts",
            "rbf_debug_inner_matvec", "rbf_set_option", "rbf_store_f64_bytes"]

RBF_OPT_FUSED_STEP, RBF_OPT_SYMMETRIC_F32, RBF_OPT_BARRIER_SPIN_LIMIT, RBF_OPT_BARRIER_EXTRA_BLOCK = 1, 2, 3, 4
RBF_OPT_SYMMETRIC_F64 = 5
RBF_OPT_STREAM_GS, RBF_OPT_STREAM_WAIT_CHECK, RBF_OPT_STORE_F64 = 6, 7, 8

RBF_PROF_MATVEC_F64, RBF_PROF_MATVEC_F32, RBF_PROF_RASM_APPLY, RBF_PROF_ORTHO, RBF_PROF_RASM_SETUP, RBF_PROF_BIN, \
    RBF_PROF_STORE_F64 = range(7)
RBF_PROF_COUNT = 7


class RbfParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("cutoff", C.c_double), ("cell_size", C.c_double), ("normalized", C.c_int),
                ("tile_f64", C.c_int), ("tile_f32", C.c_int)]


class RbfRasmParams(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("core_size", C.c_double), ("overlap", C.c_double),
                ("max_sub_points", C.c_int), ("precision", C.c_int), ("additive", C.c_int)]


class RbfSolveParams(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int), ("max_iters", C.c_int), ("mixed", C.c_int),
                ("max_refine", C.c_int), ("inner_rtol", C.c_double), ("inner_cutoff", C.c_double)]


class RbfSolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("refinements", C.c_int), ("relres", C.c_double),
                ("relres_est", C.c_double), ("matvecs", C.c_int), ("applies", C.c_int), ("status", C.c_int),
                ("stagnated", C.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class RbfServerParams(C.Structure):
    _fields_ = [("device", C.c_int), ("slots", C.c_int), ("mem_budget", C.c_int64)]


class RbfRequest(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("f", C.c_void_p), ("w", C.c_void_p), ("n", C.c_int64),
                ("kernel", RbfParams), ("rasm", RbfRasmParams), ("solve", RbfSolveParams)]


class RbfRequestResult(C.Structure):
    _fields_ = [("info", RbfSolveInfo), ("status", C.c_int), ("slot", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("footprint", C.c_int64)]


class RbfServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("resident_bytes", C.c_int64), ("mem_budget", C.c_int64), ("peak_resident_bytes", C.c_int64),
                ("trims", C.c_int64), ("launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class RbfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load librbf.so (built by ``paper_0909_5413_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"librbf.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    P, D, I32, I64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    L.rbf_create.argtypes = [C.POINTER(P), C.c_int]
    L.rbf_destroy.argtypes = [P]
    L.rbf_destroy.restype = None
    L.rbf_bin.argtypes = [P, P, C.c_int64, C.POINTER(RbfParams), P]
    L.rbf_matvec.argtypes = [P, P, P, C.c_int, P]
    L.rbf_rasm_setup.argtypes = [P, C.POINTER(RbfRasmParams), P]
    L.rbf_rasm_apply.argtypes = [P, P, P, P]
    L.rbf_rasm_factor_counts.argtypes = [P, I64, I64]
    L.rbf_solve.argtypes = [P, P, P, C.POINTER(RbfSolveParams), C.POINTER(RbfSolveInfo), P]
    L.rbf_interpolate_host.argtypes = [P, P, P, P, C.c_int64, C.POINTER(RbfParams), C.POINTER(RbfRasmParams),
                                       C.POINTER(RbfSolveParams), C.POINTER(RbfSolveInfo), P]
    L.rbf_get_grid.argtypes = [P, I64, I64, D]
    L.rbf_get_bins.argtypes = [P, P, P, P]
    L.rbf_get_subdomain_sizes.argtypes = [P, I64, I64, I64, I64]
    L.rbf_get_subdomains.argtypes = [P, P, P, P, P, P]
    L.rbf_count_neighbors.argtypes = [P, I64, P]
    L.rbf_count_candidates.argtypes = [P, C.c_int, I64, P]
    L.rbf_count_pairs.argtypes = [P, C.c_int, I64, P]
    L.rbf_profile_classes.argtypes = [P, C.c_uint]
    L.rbf_get_neighbors.argtypes = [P, P, P, C.c_int64, P]
    L.rbf_status_string.argtypes = [C.c_int]
    L.rbf_status_string.restype = C.c_char_p
    L.rbf_last_error.argtypes = [P]
    L.rbf_last_error.restype = C.c_char_p
    L.rbf_launch_count.argtypes = [P]
    L.rbf_launch_count.restype = C.c_uint64
    L.rbf_device_bytes.argtypes = [P]
    L.rbf_device_bytes.restype = C.c_int64
    L.rbf_store_f64_bytes.argtypes = [P]
    L.rbf_store_f64_bytes.restype = C.c_int64
    L.rbf_set_memory_limit.argtypes = [P, C.c_int64]
    L.rbf_set_option.argtypes = [P, C.c_int, C.c_int64]
    L.rbf_profile_enable.argtypes = [P, C.c_int]
    L.rbf_profile_read.argtypes = [P, C.c_int, I64, D]
    L.rbf_debug_exp.argtypes = [P, P, P, C.c_int64, C.c_int, P]
    L.rbf_matvec_noalloc.argtypes = [P, P, P, P]
    L.rbf_debug_kernel_pairs.argtypes = [P, P, P, C.c_int64, P]
    L.rbf_debug_inner_matvec.argtypes = [P, C.c_double, P, P, C.c_int, P]
    L.rbf_eval.argtypes = [P, P, C.c_int64, P, P, P]
    L.rbf_tune.argtypes = [P, P, C.c_int64, C.POINTER(RbfParams), C.c_double, C.c_double, C.POINTER(RbfParams),
                           C.POINTER(C.c_double), P]
    L.rbf_bin_batch.argtypes = [P, P, I64, C.c_int64, C.POINTER(RbfParams), P]
    L.rbf_rasm_setup_batch.argtypes = [P, C.POINTER(RbfRasmParams), P]
    L.rbf_solve_batch.argtypes = [P, P, P, C.POINTER(RbfSolveParams), C.POINTER(RbfSolveInfo), P]
    L.rbf_server_create.argtypes = [C.POINTER(P), C.POINTER(RbfServerParams)]
    L.rbf_server_destroy.argtypes = [P]
    L.rbf_server_destroy.restype = None
    L.rbf_server_submit.argtypes = [P, C.POINTER(RbfRequest), I64]
    L.rbf_server_wait.argtypes = [P, C.c_int64, C.c_double, C.POINTER(RbfRequestResult)]
    L.rbf_server_get_stats.argtypes = [P, C.POINTER(RbfServerStats)]
    L.rbf_server_clock.argtypes = [P]
    L.rbf_server_clock.restype = C.c_double
    L.rbf_request_footprint.argtypes = [C.POINTER(RbfRequest)]
    L.rbf_request_footprint.restype = C.c_int64
    for name in EXPORTED:
        if name not in ("rbf_destroy", "rbf_status_string", "rbf_last_error", "rbf_launch_count",
                        "rbf_device_bytes", "rbf_store_f64_bytes", "rbf_server_destroy", "rbf_server_clock",
                        "rbf_request_footprint"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(t) -> C.c_void_p:
    """Raw device (or host) pointer of a tensor / numpy array / int."""
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, int):
        return C.c_void_p(t)
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def _stream(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _check(ctx, st: int) -> int:
    if st != 0:
        L = load()
        msg = L.rbf_last_error(ctx).decode() if ctx else ""
        raise RbfError(st, msg or L.rbf_status_string(st).decode())
    return st


def rbf_create(device: int = 0) -> C.c_void_p:
    L = load()
    h = C.c_void_p()
    st = L.rbf_create(C.byref(h), int(device))
    if st != 0:
        raise RbfError(st, f"rbf_create(device={device}) failed")
    return h


def rbf_destroy(ctx) -> None:
    load().rbf_destroy(ctx)


def rbf_bin(ctx, xy_dev, n: int, params: RbfParams, stream=None) -> None:
    _check(ctx, load().rbf_bin(ctx, _ptr(xy_dev), int(n), C.byref(params), _stream(stream)))


def rbf_matvec(ctx, w_dev, y_dev, precision: int = RBF_FP64, stream=None) -> None:
    _check(ctx, load().rbf_matvec(ctx, _ptr(w_dev), _ptr(y_dev), int(precision), _stream(stream)))


def rbf_eval(ctx, xe_dev, m: int, w_dev, s_dev, stream=None) -> None:
    _check(ctx, load().rbf_eval(ctx, _ptr(xe_dev), int(m), _ptr(w_dev), _ptr(s_dev), _stream(stream)))


def rbf_tune(ctx, xy_dev, n: int, base: RbfParams, w_f64: float = 1.0, w_f32: float = 0.0,
             stream=None) -> tuple[RbfParams, float]:
    """Autotuned cell size and matvec tiles; the context is left binned with them."""
    best = RbfParams()
    score = C.c_double()
    _check(ctx, load().rbf_tune(ctx, _ptr(xy_dev), int(n), C.byref(base), float(w_f64), float(w_f32), C.byref(best),
                                C.byref(score), _stream(stream)))
    return best, score.value


def rbf_matvec_noalloc(ctx, w_dev, y_dev, stream=None) -> None:
    """FP64 matvec that allocates nothing (static device scratch, n <= 2^20)."""
    _check(ctx, load().rbf_matvec_noalloc(ctx, _ptr(w_dev), _ptr(y_dev), _stream(stream)))


def rbf_rasm_setup(ctx, params: RbfRasmParams, stream=None) -> None:
    _check(ctx, load().rbf_rasm_setup(ctx, C.byref(params), _stream(stream)))


def rbf_rasm_factor_counts(ctx) -> tuple[int, int]:
    """(subdomains inverted on the tensor cores, subdomains inverted in FP64) at the last setup."""
    tc, f64 = C.c_int64(), C.c_int64()
    _check(ctx, load().rbf_rasm_factor_counts(ctx, C.byref(tc), C.byref(f64)))
    return tc.value, f64.value


def rbf_rasm_apply(ctx, r_dev, z_dev, stream=None) -> None:
    _check(ctx, load().rbf_rasm_apply(ctx, _ptr(r_dev), _ptr(z_dev), _stream(stream)))


def rbf_solve(ctx, f_dev, w_dev, params: RbfSolveParams, stream=None, check: bool = True) -> tuple[int, RbfSolveInfo]:
    info = RbfSolveInfo()
    st = load().rbf_solve(ctx, _ptr(f_dev), _ptr(w_dev), C.byref(params), C.byref(info), _stream(stream))
    if check:
        _check(ctx, st)
    return st, info


def rbf_interpolate_host(ctx, xy_host, f_host, w_host, n: int, params: RbfParams, rasm: RbfRasmParams,
                         solve: RbfSolveParams, stream=None, check: bool = True) -> tuple[int, RbfSolveInfo]:
    info = RbfSolveInfo()
    st = load().rbf_interpolate_host(ctx, _ptr(xy_host), _ptr(f_host), _ptr(w_host), int(n), C.byref(params),
                                     C.byref(rasm), C.byref(solve), C.byref(info), _stream(stream))
    if check:
        _check(ctx, st)
    return st, info


def rbf_bin_batch(ctx, xy_dev, ptr, params, stream=None) -> None:
    """``ptr`` (nprob + 1 offsets) and ``params`` may be lists or ctypes arrays
    (``batch_ctypes``); arrays are passed without copying."""
    nprob = len(params)
    p = ptr if isinstance(ptr, C.Array) else (C.c_int64 * (nprob + 1))(*[int(v) for v in ptr])
    pa = params if isinstance(params, C.Array) else (RbfParams * nprob)(*params)
    _check(ctx, load().rbf_bin_batch(ctx, _ptr(xy_dev), p, nprob, pa, _stream(stream)))


def rbf_rasm_setup_batch(ctx, params, stream=None) -> None:
    pa = params if isinstance(params, C.Array) else (RbfRasmParams * len(params))(*params)
    _check(ctx, load().rbf_rasm_setup_batch(ctx, pa, _stream(stream)))


def rbf_solve_batch(ctx, f_dev, w_dev, params: RbfSolveParams, nprob: int, stream=None,
                    check: bool = True) -> tuple[int, list[RbfSolveInfo]]:
    infos = (RbfSolveInfo * nprob)()
    st = load().rbf_solve_batch(ctx, _ptr(f_dev), _ptr(w_dev), C.byref(params), infos, _stream(stream))
    if check:
        _check(ctx, st)
    return st, list(infos)


def rbf_get_grid(ctx) -> tuple[int, int, tuple[float, float, float, float]]:
    ncx, ncy = C.c_int64(), C.c_int64()
    bbox = (C.c_double * 4)()
    _check(ctx, load().rbf_get_grid(ctx, C.byref(ncx), C.byref(ncy), bbox))
    return ncx.value, ncy.value, tuple(bbox)


def rbf_get_bins(ctx, perm_dev, cell_start_dev, stream=None) -> None:
    _check(ctx, load().rbf_get_bins(ctx, _ptr(perm_dev), _ptr(cell_start_dev), _stream(stream)))


def rbf_get_subdomain_sizes(ctx) -> tuple[int, int, int, int]:
    v = [C.c_int64() for _ in range(4)]
    _check(ctx, load().rbf_get_subdomain_sizes(ctx, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def rbf_get_subdomains(ctx, core_ptr, core_idx, ov_ptr, ov_idx, stream=None) -> None:
    _check(ctx, load().rbf_get_subdomains(ctx, _ptr(core_ptr), _ptr(core_idx), _ptr(ov_ptr), _ptr(ov_idx),
                                          _stream(stream)))


def rbf_count_neighbors(ctx, stream=None) -> int:
    t = C.c_int64()
    _check(ctx, load().rbf_count_neighbors(ctx, C.byref(t), _stream(stream)))
    return t.value


def rbf_count_candidates(ctx, grid: int = 0, stream=None) -> int:
    """Candidate pairs of the FP32 matvec on grid 0 (cells of side r_c) or 1 (the mixed form's inner grid)."""
    t = C.c_int64()
    _check(ctx, load().rbf_count_candidates(ctx, int(grid), C.byref(t), _stream(stream)))
    return t.value


def rbf_count_pairs(ctx, grid: int = 0, stream=None) -> int:
    """Pairs within r_c (grid 0) or within the mixed form's inner cutoff (grid 1)."""
    t = C.c_int64()
    _check(ctx, load().rbf_count_pairs(ctx, int(grid), C.byref(t), _stream(stream)))
    return t.value


def rbf_get_neighbors(ctx, ptr_dev, idx_dev, capacity: int, stream=None) -> None:
    _check(ctx, load().rbf_get_neighbors(ctx, _ptr(ptr_dev), _ptr(idx_dev), int(capacity), _stream(stream)))


def rbf_launch_count(ctx) -> int:
    return int(load().rbf_launch_count(ctx))


def rbf_device_bytes(ctx) -> int:
    return int(load().rbf_device_bytes(ctx))


def rbf_store_f64_bytes(ctx) -> int:
    """Bytes of the FP64 pair values and masks kept for the current binning (0: none)."""
    return int(load().rbf_store_f64_bytes(ctx))


def rbf_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, load().rbf_set_option(ctx, int(option), int(value)))


def rbf_set_memory_limit(ctx, nbytes: int) -> None:
    """Cap on the device bytes the context may hold (0 = none)."""
    _check(ctx, load().rbf_set_memory_limit(ctx, int(nbytes)))


def rbf_profile_enable(ctx, enable: bool = True) -> None:
    _check(ctx, load().rbf_profile_enable(ctx, int(enable)))


def rbf_profile_classes(ctx, mask: int) -> None:
    """Kernel classes recorded while profiling is on (bit k = class k)."""
    _check(ctx, load().rbf_profile_classes(ctx, int(mask) & 0xFFFFFFFF))


def rbf_profile_read(ctx, kernel: int) -> tuple[int, float]:
    n, ms = C.c_int64(), C.c_double()
    _check(ctx, load().rbf_profile_read(ctx, int(kernel), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def rbf_debug_exp(ctx, t_dev, out_dev, variant: int = 0, stream=None) -> None:
    _check(ctx, load().rbf_debug_exp(ctx, _ptr(t_dev), _ptr(out_dev), t_dev.numel(), int(variant), _stream(stream)))


def rbf_debug_inner_matvec(ctx, inner_cutoff: float, w_dev, y_dev, variant: int = 0, stream=None) -> None:
    """The mixed form's FP32 inner operator (variant 0 symmetric kernel, 1 stencil kernel)."""
    _check(ctx, load().rbf_debug_inner_matvec(ctx, float(inner_cutoff), _ptr(w_dev), _ptr(y_dev), int(variant),
                                              _stream(stream)))


def rbf_debug_kernel_pairs(ctx, pairs_dev, out_dev, stream=None) -> None:
    _check(ctx, load().rbf_debug_kernel_pairs(ctx, _ptr(pairs_dev), _ptr(out_dev), out_dev.numel(), _stream(stream)))


def rbf_status_string(status: int) -> str:
    return load().rbf_status_string(int(status)).decode()


# --------------------------------------------------------------- convenience

@dataclasses.dataclass
class SolverConfig:
    sigma: float
    cutoff: float
    x0: float
    y0: float
    core_size: float
    overlap: float
    cell_size: float = 0.0
    tile_f64: int = 0               # targets per block of the FP64 / FP32 matvecs (0 = 128)
    tile_f32: int = 0
    normalized: bool = False
    max_sub_points: int = 0
    factor_precision: int = RBF_FP64
    additive: bool = False          # Eq. asm instead of Eq. rasm
    rtol: float = 1e-13
    restart: int = 30
    max_iters: int = 10000
    mixed: bool = False
    max_refine: int = 40
    inner_rtol: float = 1e-5
    inner_cutoff: float = 0.0       # mixed only: shorter cutoff (in sigma) of the FP32 inner grid; 0 = r_c

    def params(self) -> RbfParams:
        return RbfParams(self.sigma, self.cutoff, self.cell_size, int(self.normalized), self.tile_f64, self.tile_f32)

    def rasm(self) -> RbfRasmParams:
        return RbfRasmParams(self.x0, self.y0, self.core_size, self.overlap, self.max_sub_points,
                             self.factor_precision, int(self.additive))

    def solve(self) -> RbfSolveParams:
        return RbfSolveParams(self.rtol, self.restart, self.max_iters, int(self.mixed), self.max_refine,
                              self.inner_rtol, self.inner_cutoff)


class Context:
    """Owns one ``rbf_ctx``; methods forward to the C entry points."""

    def __init__(self, device: int = 0):
        self.handle = rbf_create(device)
        self.device = device

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            rbf_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bin(self, xy_dev, cfg: SolverConfig, stream=None) -> None:
        rbf_bin(self.handle, xy_dev, xy_dev.shape[0], cfg.params(), stream)

    def matvec(self, w_dev, y_dev, precision: int = RBF_FP64, stream=None) -> None:
        rbf_matvec(self.handle, w_dev, y_dev, precision, stream)

    def rasm_setup(self, cfg: SolverConfig, stream=None) -> None:
        rbf_rasm_setup(self.handle, cfg.rasm(), stream)

    def rasm_apply(self, r_dev, z_dev, stream=None) -> None:
        rbf_rasm_apply(self.handle, r_dev, z_dev, stream)

    def solve(self, f_dev, w_dev, cfg: SolverConfig, stream=None, check: bool = True):
        return rbf_solve(self.handle, f_dev, w_dev, cfg.solve(), stream, check)

    def interpolate_host(self, xy_host, f_host, w_host, cfg: SolverConfig, stream=None, check: bool = True):
        return rbf_interpolate_host(self.handle, xy_host, f_host, w_host, xy_host.shape[0], cfg.params(),
                                    cfg.rasm(), cfg.solve(), stream, check)

    @property
    def launches(self) -> int:
        return rbf_launch_count(self.handle)


def batch_arrays(problems, cell_size: float = 0.0, factor_precision: int = RBF_FP64, max_sub_points: int = 0):
    """Concatenated inputs of a batch: (xy (N, 2), f (N,), ptr, [RbfParams], [RbfRasmParams])."""
    import numpy as np
    xy = np.ascontiguousarray(np.concatenate([p.xy for p in problems]), dtype=np.float64)
    f = np.ascontiguousarray(np.concatenate([p.f for p in problems]), dtype=np.float64)
    ptr = [0]
    for p in problems:
        ptr.append(ptr[-1] + p.n)
    params = [RbfParams(p.sigma, p.cutoff, cell_size, 0) for p in problems]
    rasm = [RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, max_sub_points, factor_precision) for p in problems]
    return xy, f, ptr, params, rasm


def batch_ctypes(ptr, params, rasm):
    """The per-problem tables of ``batch_arrays`` as ctypes arrays, built once."""
    n = len(params)
    return ((C.c_int64 * (n + 1))(*[int(v) for v in ptr]), (RbfParams * n)(*params), (RbfRasmParams * n)(*rasm))


def config_for(problem, **kw) -> SolverConfig:
    """SolverConfig from a ``workloads.Problem``."""
    return SolverConfig(sigma=problem.sigma, cutoff=problem.cutoff, x0=problem.x0, y0=problem.x0,
                        core_size=problem.core_size, overlap=problem.overlap, **kw)


# ---------------------------------------------------------------- serving

def rbf_server_create(device: int = 0, slots: int = 4, mem_budget: int = 0):
    h = C.c_void_p()
    p = RbfServerParams(device, slots, mem_budget)
    st = load().rbf_server_create(C.byref(h), C.byref(p))
    if st != 0:
        raise RbfError(st, "rbf_server_create")
    return h


def rbf_server_destroy(server) -> None:
    load().rbf_server_destroy(server)


def rbf_server_submit(server, req: RbfRequest) -> int:
    t = C.c_int64()
    st = load().rbf_server_submit(server, C.byref(req), C.byref(t))
    if st != 0:
        raise RbfError(st, "rbf_server_submit")
    return t.value


def rbf_server_wait(server, ticket: int, timeout_s: float = -1.0) -> tuple[int, RbfRequestResult]:
    r = RbfRequestResult()
    st = load().rbf_server_wait(server, int(ticket), float(timeout_s), C.byref(r))
    return st, r


def rbf_server_get_stats(server) -> RbfServerStats:
    s = RbfServerStats()
    st = load().rbf_server_get_stats(server, C.byref(s))
    if st != 0:
        raise RbfError(st, "rbf_server_get_stats")
    return s


def rbf_server_clock(server) -> float:
    return float(load().rbf_server_clock(server))


def rbf_request_footprint(req: RbfRequest) -> int:
    return int(load().rbf_request_footprint(C.byref(req)))


def make_request(xy, f, w, cfg: SolverConfig) -> RbfRequest:
    """Request over host arrays (C-contiguous float64 numpy arrays; xy (n, 2))."""
    n = int(f.shape[0])
    return RbfRequest(_ptr(xy), _ptr(f), _ptr(w), n, cfg.params(), cfg.rasm(), cfg.solve())


class Server:
    """Owns one ``rbf_server``; keeps each request's host arrays alive until
    its result has been collected."""

    def __init__(self, device: int = 0, slots: int = 4, mem_budget: int = 0):
        self.handle = rbf_server_create(device, slots, mem_budget)
        self._live: dict[int, tuple] = {}

    def submit(self, xy, f, cfg: SolverConfig, w=None) -> int:
        import numpy as np
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        if w is None:
            w = np.zeros(f.shape[0], dtype=np.float64)
        req = make_request(xy, f, w, cfg)
        t = rbf_server_submit(self.handle, req)
        self._live[t] = (xy, f, w)
        return t

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """(status of the wait, RbfRequestResult, w) -- w is None on a timeout."""
        st, r = rbf_server_wait(self.handle, ticket, timeout_s)
        if st != 0:
            return st, r, None
        _, _, w = self._live.pop(ticket)
        return st, r, w

    def stats(self) -> dict:
        return rbf_server_get_stats(self.handle).as_dict()

    def clock(self) -> float:
        return rbf_server_clock(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            rbf_server_destroy(self.handle)
            self.handle = C.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
