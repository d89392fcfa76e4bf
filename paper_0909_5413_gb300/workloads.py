"""Seeded synthetic inputs for the Gaussian RBF interpolation problem.

This module only draws points and right-hand sides; it holds none of the
solver's arithmetic, and both the CUDA path and the CPU oracle consume the
arrays it returns (so the two never see different input bits).

Workloads (all coordinates FP64, AoS ``(N, 2)``, user order = row-major
lattice order ``j * n + i``):

* jittered lattice on [-1, 1]^2: ``n`` points per side at spacing
  ``h = 2 / (n - 1)`` (inclusive end points, the point-count convention
  ``N = (1/h + 1)^2`` of Sec. 3.1 scaled to a side of 2), each coordinate
  moved by an independent U(-0.1 h, +0.1 h) draw;
* Gaussian width ``sigma = h / ratio`` (``ratio = h / sigma``; 0.8 for the
  plain and mixed workloads), cutoff ``r_c = 8.6 sigma``;
* RASM boxes of 4 x 4 lattice points with a ring of one lattice point:
  ``B = 4 h``, ``delta = h``, box origin ``-1 - h/2`` so that box edges lie
  on lattice mid-lines;
* right-hand sides: ``exp(-|x|^2 / 0.1) + 0.1 sin(4 pi x) cos(4 pi y)``;
  Franke's test function (Sec. 3.1); or a sum of four Gaussians with random
  amplitudes, centres and widths for the many-problem workloads.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEFAULT_SEED = 20250909


@dataclasses.dataclass(frozen=True)
class Problem:
    """One interpolation problem: points, right-hand side and parameters."""

    name: str
    xy: np.ndarray          # (N, 2) float64, C-contiguous
    f: np.ndarray           # (N,) float64
    n_side: int
    h: float
    sigma: float
    cutoff: float
    x0: float               # RASM box origin (both axes)
    core_size: float        # B
    overlap: float          # delta
    seed: int

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])


def jittered_lattice(n_side: int, seed: int, jitter: float = 0.1,
                     lo: float = -1.0, hi: float = 1.0) -> tuple[np.ndarray, float]:
    """``n_side^2`` points on a lattice over [lo, hi]^2 with U(-jitter h, jitter h)
    per coordinate. Returns ``(xy, h)``."""
    if n_side < 1:
        raise ValueError("n_side must be >= 1")
    h = (hi - lo) / (n_side - 1) if n_side > 1 else (hi - lo)
    g = lo + h * np.arange(n_side, dtype=np.float64)
    xs, ys = np.meshgrid(g, g, indexing="xy")  # xs varies fastest along a row
    xy = np.stack([xs.ravel(), ys.ravel()], axis=1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        xy = xy + rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    return np.ascontiguousarray(xy, dtype=np.float64), h


def rhs_gauss_sincos(xy: np.ndarray) -> np.ndarray:
    x, y = xy[:, 0], xy[:, 1]
    return np.exp(-(x * x + y * y) / 0.1) + 0.1 * np.sin(4 * np.pi * x) * np.cos(4 * np.pi * y)


def rhs_franke(xy: np.ndarray) -> np.ndarray:
    """Franke's bivariate test function (Sec. 3.1), defined on [0, 1]^2."""
    return _franke_terms(xy[:, 0], xy[:, 1])


def franke(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Franke's function at arbitrary points (x, y arrays)."""
    return _franke_terms(x, y)


def _franke_terms(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    t1 = 0.75 * np.exp(-0.25 * ((9 * x - 2) ** 2 + (9 * y - 2) ** 2))
    # Sec. 3.1 prints the second term's y part squared, -(9y+1)^2/10; that
    # printed form is what is used here.
    t2 = 0.75 * np.exp(-((9 * x + 1) ** 2) / 49.0 - ((9 * y + 1) ** 2) / 10.0)
    t3 = 0.5 * np.exp(-0.25 * ((9 * x - 7) ** 2 + (9 * y - 3) ** 2))
    t4 = -0.2 * np.exp(-((9 * x - 4) ** 2) - (9 * y - 7) ** 2)
    return t1 + t2 + t3 + t4


def rhs_four_gaussians(xy: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Sum of 4 Gaussians: amplitudes U[-1,1], centres U[-1,1]^2, widths U[0.1, 0.5]."""
    a = rng.uniform(-1.0, 1.0, size=4)
    c = rng.uniform(-1.0, 1.0, size=(4, 2))
    s = rng.uniform(0.1, 0.5, size=4)
    out = np.zeros(xy.shape[0])
    for k in range(4):
        d2 = (xy[:, 0] - c[k, 0]) ** 2 + (xy[:, 1] - c[k, 1]) ** 2
        out += a[k] * np.exp(-d2 / (2.0 * s[k] * s[k]))
    return out


def lattice_problem(n_side: int, ratio: float = 0.8, seed: int = DEFAULT_SEED,
                    rhs: str = "gauss_sincos", cutoff_sigmas: float = 8.6,
                    core_points: int = 4, ring_points: int = 1,
                    jitter: float = 0.1, name: str | None = None) -> Problem:
    """Jittered lattice on [-1, 1]^2 with ``sigma = h / ratio`` (see module doc)."""
    xy, h = jittered_lattice(n_side, seed, jitter)
    sigma = h / ratio
    if rhs == "gauss_sincos":
        f = rhs_gauss_sincos(xy)
    elif rhs == "four_gaussians":
        f = rhs_four_gaussians(xy, np.random.default_rng(seed + 7919))
    else:
        raise ValueError(rhs)
    return Problem(name=name or f"lattice{n_side}_r{ratio}_s{seed}", xy=xy, f=np.ascontiguousarray(f),
                   n_side=n_side, h=h, sigma=sigma, cutoff=cutoff_sigmas * sigma,
                   x0=-1.0 - 0.5 * h, core_size=core_points * h, overlap=ring_points * h, seed=seed)


def config_small(seed: int = DEFAULT_SEED) -> Problem:
    """64 x 64 jittered lattice, h/sigma = 0.8 (N = 4,096)."""
    return lattice_problem(64, 0.8, seed, name="lattice64_f64")


def config_1m(seed: int = DEFAULT_SEED) -> Problem:
    """1024 x 1024 jittered lattice, h/sigma = 0.8 (N = 1,048,576)."""
    return lattice_problem(1024, 0.8, seed, name="lattice1024_f64")


def config_4m(seed: int = DEFAULT_SEED) -> Problem:
    """2048 x 2048 jittered lattice, h/sigma = 0.8 (N = 4,194,304): above the L2 cache, small
    enough for detailed kernel captures."""
    return lattice_problem(2048, 0.8, seed, name="lattice2048")


def config_51m(seed: int = DEFAULT_SEED) -> Problem:
    """7168 x 7168 jittered lattice, h/sigma = 0.8 (N = 51,380,224)."""
    return lattice_problem(7168, 0.8, seed, name="lattice7168")


def batch_problem_sizes(count: int, lo: int, hi: int, seed: int) -> list[tuple[int, float]]:
    """Per-problem ``(n_side, ratio)`` for the many-problem workloads: N log-uniform
    in [lo, hi] (``n_side = round(sqrt(N))``), h/sigma uniform in [0.6, 1.0]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        out.append((max(2, int(round(math.sqrt(n)))), float(rng.uniform(0.6, 1.0))))
    return out


def batch_workload(count: int, lo: int = 256, hi: int = 16384, seed: int = DEFAULT_SEED,
                   ratio_lo: float = 0.6, ratio_hi: float = 1.0) -> list[Problem]:
    """Many independent problems: N log-uniform in [lo, hi] (n_side = round(sqrt N)),
    h/sigma uniform in [ratio_lo, ratio_hi], each on its own jittered lattice over
    [-1, 1]^2 with a sum of four random Gaussians as right-hand side; problem k
    uses seed + k."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        n_side = max(2, int(round(math.sqrt(n))))
        ratio = float(rng.uniform(ratio_lo, ratio_hi))
        out.append(lattice_problem(n_side, ratio, seed=seed + 1 + k, rhs="four_gaussians",
                                   name=f"batch{k}_n{n_side}_r{ratio:.3f}"))
    return out


def unit_square_problem(h_over_sigma: float, sigma: float = 0.01, seed: int = DEFAULT_SEED,
                        jitter: float = 0.0) -> Problem:
    """Franke's function on a lattice over [0, 1]^2 with ``N = (1/h + 1)^2`` (Sec. 3.1),
    paper subdomain sizes B = 5 sigma, D = 1.9 B (delta = 0.45 B)."""
    h = h_over_sigma * sigma
    n_side = int(round(1.0 / h)) + 1
    xy, h2 = jittered_lattice(n_side, seed, jitter, lo=0.0, hi=1.0)
    f = _franke_terms(xy[:, 0], xy[:, 1])
    B = 5.0 * sigma
    return Problem(name=f"unit{n_side}_r{h_over_sigma}", xy=xy, f=np.ascontiguousarray(f), n_side=n_side,
                   h=h2, sigma=sigma, cutoff=8.6 * sigma, x0=-0.5 * h2, core_size=B,
                   overlap=0.45 * B, seed=seed)
