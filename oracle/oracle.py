"""ctypes front end of the C oracle (``rbf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the product path never does. It
imports nothing from the CUDA package.

All vectors are in the caller's (original) point order, FP64.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


class OrcKernelParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("rc", C.c_double), ("normalized", C.c_int)]


class OrcGrid(C.Structure):
    _fields_ = [("xmin", C.c_double), ("ymin", C.c_double), ("xmax", C.c_double), ("ymax", C.c_double),
                ("c", C.c_double), ("ncx", C.c_int64), ("ncy", C.c_int64)]


class OrcBoxes(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("B", C.c_double), ("delta", C.c_double),
                ("nbx", C.c_int64), ("nby", C.c_int64)]


class OrcGmresInfo(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("relres", C.c_double), ("status", C.c_int)]


OP = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_kernel.restype = C.c_double
        L.orc_kernel.argtypes = [C.c_double, C.POINTER(OrcKernelParams)]
        L.orc_pair_r2.restype = C.c_double
        L.orc_pair_r2.argtypes = [_D, C.c_int64, C.c_int64]
        L.orc_grid_dims.argtypes = [_D, C.c_int64, C.c_double, C.POINTER(OrcGrid)]
        L.orc_bin.argtypes = [_D, C.c_int64, C.POINTER(OrcGrid), _I32, _I32]
        L.orc_stencil.restype = C.c_int64
        L.orc_stencil.argtypes = [C.c_double, C.c_double]
        L.orc_neighbor_counts.argtypes = [_D, C.c_int64, C.POINTER(OrcGrid), _I32, _I32, C.c_double, _I64]
        L.orc_neighbors.argtypes = [_D, C.c_int64, C.POINTER(OrcGrid), _I32, _I32, C.c_double, _I64, _I32]
        L.orc_matvec_cutoff.argtypes = [_D, C.c_int64, C.POINTER(OrcGrid), _I32, _I32,
                                        C.POINTER(OrcKernelParams), _D, _D]
        L.orc_matvec_dense.argtypes = [_D, C.c_int64, C.POINTER(OrcKernelParams), _D, _D]
        L.orc_eval.argtypes = [_D, C.c_int64, C.POINTER(OrcKernelParams), _D, _D, C.c_int64, _D]
        L.orc_cholesky.argtypes = [_D, C.c_int64]
        L.orc_cholesky_solve.argtypes = [_D, C.c_int64, _D]
        L.orc_dense_solve.argtypes = [_D, C.c_int64, C.POINTER(OrcKernelParams), _D, _D]
        L.orc_box_dims.argtypes = [C.POINTER(OrcGrid), C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(OrcBoxes)]
        L.orc_subdomains.argtypes = [_D, C.c_int64, C.POINTER(OrcBoxes), _I64, _I32, _I64, _I32]
        L.orc_gmres.argtypes = [C.c_int64, OP, C.c_void_p, OP, C.c_void_p, _D, _D, C.c_int64, C.c_double,
                                C.c_int64, _D, C.POINTER(OrcGmresInfo)]
        L.orc_problem_create.argtypes = [C.POINTER(C.c_void_p), _D, C.c_int64, C.c_double, C.c_double, C.c_int,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64]
        L.orc_problem_destroy.argtypes = [C.c_void_p]
        L.orc_problem_grid.argtypes = [C.c_void_p, C.POINTER(OrcGrid), C.POINTER(OrcBoxes)]
        for name, rt in [("orc_problem_perm", _I32), ("orc_problem_cell_start", _I32),
                         ("orc_problem_core_ptr", _I64), ("orc_problem_core_idx", _I32),
                         ("orc_problem_ov_ptr", _I64), ("orc_problem_ov_idx", _I32)]:
            getattr(L, name).restype = rt
            getattr(L, name).argtypes = [C.c_void_p]
        L.orc_problem_matvec.argtypes = [C.c_void_p, _D, _D]
        L.orc_problem_set_additive.argtypes = [C.c_void_p, C.c_int]
        L.orc_problem_set_additive.restype = None
        L.orc_problem_rasm_apply.argtypes = [C.c_void_p, _D, _D]
        L.orc_problem_solve.argtypes = [C.c_void_p, _D, _D, C.c_int64, C.c_double, C.c_int64, C.c_int, _D,
                                        C.POINTER(OrcGmresInfo)]
        L.orc_problem_counts.restype = C.c_int64
        L.orc_problem_counts.argtypes = [C.c_void_p, C.c_int64]
        _lib = L
    return _lib


STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 4: "subdomain matrix not SPD",
          5: "too large", 6: "not converged"}


class OracleError(RuntimeError):
    pass


def _check(st: int) -> None:
    if st:
        raise OracleError(STATUS.get(st, f"status {st}"))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (results do not depend on it)."""
    os.environ["OMP_NUM_THREADS"] = str(n)
    try:
        libgomp = C.CDLL("libgomp.so.1")
        libgomp.omp_set_num_threads(C.c_int(n))
    except OSError:
        pass


def kernel(r2: float, sigma: float, rc: float = np.inf, normalized: bool = False) -> float:
    kp = OrcKernelParams(sigma, rc, int(normalized))
    return lib().orc_kernel(float(r2), C.byref(kp))


def pair_r2(xy: np.ndarray, i: int, j: int) -> float:
    xy = _f64(xy)
    return lib().orc_pair_r2(_dp(xy), i, j)


@dataclasses.dataclass
class Grid:
    xmin: float
    ymin: float
    xmax: float
    ymax: float
    c: float
    ncx: int
    ncy: int

    @property
    def ncell(self) -> int:
        return self.ncx * self.ncy


def _grid_struct(g: Grid) -> OrcGrid:
    return OrcGrid(g.xmin, g.ymin, g.xmax, g.ymax, g.c, g.ncx, g.ncy)


def grid_dims(xy: np.ndarray, c: float) -> Grid:
    xy = _f64(xy)
    g = OrcGrid()
    _check(lib().orc_grid_dims(_dp(xy), xy.shape[0], float(c), C.byref(g)))
    return Grid(g.xmin, g.ymin, g.xmax, g.ymax, g.c, g.ncx, g.ncy)


def bin_points(xy: np.ndarray, c: float) -> tuple[Grid, np.ndarray, np.ndarray]:
    """Cell binning: ``(grid, perm, cell_start)`` (perm: sorted position -> original index)."""
    xy = _f64(xy)
    g = grid_dims(xy, c)
    perm = np.empty(xy.shape[0], np.int32)
    cs = np.empty(g.ncell + 1, np.int32)
    gs = _grid_struct(g)
    _check(lib().orc_bin(_dp(xy), xy.shape[0], C.byref(gs), perm.ctypes.data_as(_I32), cs.ctypes.data_as(_I32)))
    return g, perm, cs


def stencil(rc: float, c: float) -> int:
    return int(lib().orc_stencil(float(rc), float(c)))


def neighbors(xy: np.ndarray, rc: float, c: float | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Neighbour lists (CSR over original targets, rows ascending): ``(ptr, idx)``."""
    xy = _f64(xy)
    g, perm, cs = bin_points(xy, c if c else rc)
    gs = _grid_struct(g)
    n = xy.shape[0]
    counts = np.zeros(n, np.int64)
    L = lib()
    L.orc_neighbor_counts(_dp(xy), n, C.byref(gs), perm.ctypes.data_as(_I32), cs.ctypes.data_as(_I32),
                          float(rc), counts.ctypes.data_as(_I64))
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    idx = np.empty(int(ptr[-1]), np.int32)
    L.orc_neighbors(_dp(xy), n, C.byref(gs), perm.ctypes.data_as(_I32), cs.ctypes.data_as(_I32),
                    float(rc), ptr.ctypes.data_as(_I64), idx.ctypes.data_as(_I32))
    return ptr, idx


def matvec_cutoff(xy: np.ndarray, w: np.ndarray, sigma: float, rc: float, normalized: bool = False,
                  c: float | None = None) -> np.ndarray:
    xy, w = _f64(xy), _f64(w)
    g, perm, cs = bin_points(xy, c if c else rc)
    gs = _grid_struct(g)
    kp = OrcKernelParams(sigma, rc, int(normalized))
    y = np.empty_like(w)
    lib().orc_matvec_cutoff(_dp(xy), xy.shape[0], C.byref(gs), perm.ctypes.data_as(_I32),
                            cs.ctypes.data_as(_I32), C.byref(kp), _dp(w), _dp(y))
    return y


def matvec_dense(xy: np.ndarray, w: np.ndarray, sigma: float, normalized: bool = False) -> np.ndarray:
    xy, w = _f64(xy), _f64(w)
    kp = OrcKernelParams(sigma, np.inf, int(normalized))
    y = np.empty_like(w)
    lib().orc_matvec_dense(_dp(xy), xy.shape[0], C.byref(kp), _dp(w), _dp(y))
    return y


def eval_points(xy: np.ndarray, w: np.ndarray, xe: np.ndarray, sigma: float, rc: float,
                normalized: bool = False) -> np.ndarray:
    """Interpolant s at the points xe: every centre within r_c, in index order."""
    xy, w, xe = _f64(xy), _f64(w), _f64(xe)
    kp = OrcKernelParams(sigma, rc, int(normalized))
    out = np.empty(xe.shape[0])
    lib().orc_eval(_dp(xy), xy.shape[0], C.byref(kp), _dp(w), _dp(xe), xe.shape[0], _dp(out))
    return out


def cholesky(a: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor of an SPD matrix (raises on a non-positive pivot)."""
    a = _f64(a).copy()
    n = a.shape[0]
    _check(lib().orc_cholesky(_dp(a), n))
    return np.tril(a)


def cholesky_solve(l: np.ndarray, b: np.ndarray) -> np.ndarray:
    l, x = _f64(l), _f64(b).copy()
    lib().orc_cholesky_solve(_dp(l), l.shape[0], _dp(x))
    return x


def dense_solve(xy: np.ndarray, f: np.ndarray, sigma: float, normalized: bool = False) -> np.ndarray:
    xy, f = _f64(xy), _f64(f)
    kp = OrcKernelParams(sigma, np.inf, int(normalized))
    w = np.empty_like(f)
    _check(lib().orc_dense_solve(_dp(xy), xy.shape[0], C.byref(kp), _dp(f), _dp(w)))
    return w


def subdomains(xy: np.ndarray, x0: float, y0: float, B: float, delta: float
               ) -> tuple[tuple[int, int], np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """``((nbx, nby), core_ptr, core_idx, ov_ptr, ov_idx)`` with rows ascending."""
    xy = _f64(xy)
    g = grid_dims(xy, 1.0)
    gs = _grid_struct(g)
    b = OrcBoxes()
    _check(lib().orc_box_dims(C.byref(gs), x0, y0, B, delta, C.byref(b)))
    nsub = b.nbx * b.nby
    cp = np.zeros(nsub + 1, np.int64)
    op = np.zeros(nsub + 1, np.int64)
    L = lib()
    L.orc_subdomains(_dp(xy), xy.shape[0], C.byref(b), cp.ctypes.data_as(_I64), None, op.ctypes.data_as(_I64), None)
    ci = np.empty(int(cp[-1]), np.int32)
    oi = np.empty(int(op[-1]), np.int32)
    L.orc_subdomains(_dp(xy), xy.shape[0], C.byref(b), cp.ctypes.data_as(_I64), ci.ctypes.data_as(_I32),
                     op.ctypes.data_as(_I64), oi.ctypes.data_as(_I32))
    return (int(b.nbx), int(b.nby)), cp, ci, op, oi


@dataclasses.dataclass
class GmresInfo:
    iters: int
    restarts: int
    relres: float
    status: int
    history: np.ndarray


def gmres(amul, minv, f: np.ndarray, w0: np.ndarray | None = None, m: int = 30, rtol: float = 1e-13,
          max_iters: int = 1000) -> tuple[np.ndarray, GmresInfo]:
    """The oracle's GMRES driven by Python operators ``amul(x) -> A x`` and
    ``minv(x) -> M^{-1} x`` (numpy arrays), for pins on small explicit matrices."""
    f = _f64(f)
    n = f.shape[0]
    w = np.zeros(n) if w0 is None else _f64(w0).copy()

    def wrap(fn):
        def cb(_ctx, pin, pout):
            x = np.ctypeslib.as_array(pin, shape=(n,))
            out = np.ctypeslib.as_array(pout, shape=(n,))
            out[:] = fn(x.copy())
        return OP(cb)

    a_cb, m_cb = wrap(amul), wrap(minv if minv is not None else (lambda x: x))
    hist = np.zeros(max(1, max_iters))
    info = OrcGmresInfo()
    lib().orc_gmres(n, a_cb, None, m_cb, None, _dp(f), _dp(w), m, rtol, max_iters, _dp(hist), C.byref(info))
    return w, GmresInfo(int(info.iters), int(info.restarts), float(info.relres), int(info.status),
                        hist[: int(info.iters)].copy())


class Problem:
    """Binning, subdomain lists and RASM factors for one point set (Sec. 2)."""

    def __init__(self, xy: np.ndarray, sigma: float, rc: float, x0: float, y0: float, B: float,
                 delta: float, normalized: bool = False, cell_size: float = 0.0, max_sub_points: int = 4096,
                 additive: bool = False):
        self.xy = _f64(xy)
        self.n = self.xy.shape[0]
        self.sigma, self.rc = float(sigma), float(rc)
        h = C.c_void_p()
        st = lib().orc_problem_create(C.byref(h), _dp(self.xy), self.n, self.sigma, self.rc, int(normalized),
                                      float(cell_size), float(x0), float(y0), float(B), float(delta),
                                      int(max_sub_points))
        self._h = h
        if st:
            self.close()
            raise OracleError(STATUS.get(st, f"status {st}"))
        g, b = OrcGrid(), OrcBoxes()
        lib().orc_problem_grid(h, C.byref(g), C.byref(b))
        self.grid = Grid(g.xmin, g.ymin, g.xmax, g.ymax, g.c, g.ncx, g.ncy)
        self.nbx, self.nby = int(b.nbx), int(b.nby)
        self.nsub = self.nbx * self.nby
        lib().orc_problem_set_additive(h, int(additive))   # Eq. asm instead of Eq. rasm

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            lib().orc_problem_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        self.close()

    def _arr(self, name: str, count: int) -> np.ndarray:
        p = getattr(lib(), name)(self._h)
        return np.ctypeslib.as_array(p, shape=(count,)).copy() if count else np.zeros(0)

    @property
    def perm(self) -> np.ndarray:
        return self._arr("orc_problem_perm", self.n).astype(np.int32)

    @property
    def cell_start(self) -> np.ndarray:
        return self._arr("orc_problem_cell_start", self.grid.ncell + 1).astype(np.int32)

    def core_lists(self) -> tuple[np.ndarray, np.ndarray]:
        ptr = self._arr("orc_problem_core_ptr", self.nsub + 1).astype(np.int64)
        return ptr, self._arr("orc_problem_core_idx", int(ptr[-1])).astype(np.int32)

    def overlap_lists(self) -> tuple[np.ndarray, np.ndarray]:
        ptr = self._arr("orc_problem_ov_ptr", self.nsub + 1).astype(np.int64)
        return ptr, self._arr("orc_problem_ov_idx", int(ptr[-1])).astype(np.int32)

    def matvec(self, w: np.ndarray) -> np.ndarray:
        w = _f64(w)
        y = np.empty_like(w)
        lib().orc_problem_matvec(self._h, _dp(w), _dp(y))
        return y

    def rasm_apply(self, v: np.ndarray) -> np.ndarray:
        v = _f64(v)
        z = np.empty_like(v)
        lib().orc_problem_rasm_apply(self._h, _dp(v), _dp(z))
        return z

    def solve(self, f: np.ndarray, w0: np.ndarray | None = None, m: int = 30, rtol: float = 1e-13,
              max_iters: int = 3000, precondition: bool = True) -> tuple[np.ndarray, GmresInfo]:
        f = _f64(f)
        w = np.zeros(self.n) if w0 is None else _f64(w0).copy()
        hist = np.zeros(max(1, max_iters))
        info = OrcGmresInfo()
        lib().orc_problem_solve(self._h, _dp(f), _dp(w), m, rtol, max_iters, int(precondition), _dp(hist),
                                C.byref(info))
        return w, GmresInfo(int(info.iters), int(info.restarts), float(info.relres), int(info.status),
                            hist[: int(info.iters)].copy())

    def counts(self) -> tuple[int, int]:
        return int(lib().orc_problem_counts(self._h, 0)), int(lib().orc_problem_counts(self._h, 1))
