"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute force on small inputs, numpy/LAPACK routines, invariants of
the decomposition, and GMRES properties. CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_5413_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def np_r2(xy):
    dx = xy[:, None, 0] - xy[None, :, 0]
    dy = xy[:, None, 1] - xy[None, :, 1]
    return dx * dx + dy * dy


def np_matrix(xy, sigma, rc=np.inf):
    r2 = np_r2(xy)
    a = np.exp(-r2 / (2.0 * sigma * sigma))
    a[r2 > rc * rc] = 0.0
    return a


def random_points(n, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(lo, hi, size=(n, 2)))


# ------------------------------------------------------------------ kernel

def test_kernel_closed_form():
    s = 0.37
    assert O.kernel(0.0, s) == 1.0
    # exp(-r^2 / (2 sigma^2)) at r^2 = 2 sigma^2 is 1/e
    assert O.kernel(2 * s * s, s) == pytest.approx(math.exp(-1.0), rel=1e-15)
    # largest dropped entry at r_c = 8.6 sigma: exp(-8.6^2 / 2) = exp(-36.98)
    assert O.kernel((8.6 * s) ** 2, s) == pytest.approx(math.exp(-36.98), rel=1e-13)
    # Sec. 2.3 normalisation 1/(2 pi sigma^2)
    assert O.kernel(0.0, s, normalized=True) == pytest.approx(1.0 / (2 * math.pi * s * s), rel=1e-15)
    # Table 1's form exp(-eps^2 r^2) with eps^2 = 1/(2 sigma^2)
    r = 0.81
    assert O.kernel(r * r, s) == pytest.approx(math.exp(-(r * r) / (2 * s * s)), rel=1e-14)


def test_pair_r2_rounds_each_product():
    """The oracle's squared distance must equal numpy's unfused (dx*dx)+(dy*dy)
    bit for bit: the build must not contract to FMA."""
    xy = random_points(300, 3)
    r2 = np_r2(xy)
    for i, j in [(0, 1), (5, 200), (17, 17), (299, 3), (100, 250)]:
        assert O.pair_r2(xy, i, j) == r2[i, j]
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j = rng.integers(0, 300, 2)
        assert O.pair_r2(xy, int(i), int(j)) == r2[i, j]


# ----------------------------------------------------------------- binning

def np_cells(xy, c):
    xmin, ymin = xy[:, 0].min(), xy[:, 1].min()
    ncx = int(np.floor((xy[:, 0].max() - xmin) / c)) + 1
    ncy = int(np.floor((xy[:, 1].max() - ymin) / c)) + 1
    cx = np.clip(np.floor((xy[:, 0] - xmin) / c), 0, ncx - 1).astype(np.int64)
    cy = np.clip(np.floor((xy[:, 1] - ymin) / c), 0, ncy - 1).astype(np.int64)
    return cy * ncx + cx, ncx, ncy


def binning_cases():
    p = W.config_small()
    yield "lattice64", p.xy, p.cutoff
    yield "lattice64_half", p.xy, p.cutoff / 2
    for n in (1, 2, 15, 16, 17, 255):
        yield f"rand{n}", random_points(n, n), 0.3
    yield "one_cell", random_points(200, 9, 0.0, 0.01), 1.0
    # an empty band of cells between two clusters
    a = random_points(100, 11, -1.0, -0.5)
    b = random_points(100, 12, 0.5, 1.0)
    yield "gap", np.ascontiguousarray(np.vstack([a, b])), 0.2
    # duplicates and points exactly on cell edges
    e = np.array([[0.0, 0.0], [0.25, 0.0], [0.5, 0.5], [0.25, 0.0], [0.75, 1.0], [1.0, 1.0]])
    yield "edges", e, 0.25


@pytest.mark.parametrize("name,xy,c", list(binning_cases()), ids=[x[0] for x in binning_cases()])
def test_binning_matches_numpy_stable_sort(name, xy, c):
    g, perm, cs = O.bin_points(xy, c)
    cell, ncx, ncy = np_cells(xy, c)
    assert (g.ncx, g.ncy) == (ncx, ncy)
    np.testing.assert_array_equal(perm, np.argsort(cell, kind="stable").astype(np.int32))
    counts = np.bincount(cell, minlength=ncx * ncy)
    np.testing.assert_array_equal(cs, np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    # every sorted point lies in its cell's box (up to the clamp at the top edge)
    sc = cell[perm]
    assert np.all(np.diff(sc) >= 0)


def test_stencil_width():
    assert O.stencil(1.0, 1.0) == 1
    assert O.stencil(1.0, 0.5) == 2
    assert O.stencil(1.0, 1.0 / 3.0) == 3
    assert O.stencil(1.0, 0.4) == 3


# -------------------------------------------------------------- neighbours

@pytest.mark.parametrize("cfac", [1.0, 0.5, 1.0 / 3.0, 2.0])
def test_neighbors_match_brute_force(cfac):
    p = W.lattice_problem(40, 0.8, seed=5)
    rc = p.cutoff
    ptr, idx = O.neighbors(p.xy, rc, c=rc * cfac)
    r2 = np_r2(p.xy)
    for i in range(p.n):
        ref = np.nonzero(r2[i] <= rc * rc)[0]
        np.testing.assert_array_equal(idx[ptr[i]:ptr[i + 1]], ref.astype(np.int32))


def test_neighbor_count_matches_area():
    """Inside the lattice each point sees about pi (r_c/h)^2 others."""
    p = W.lattice_problem(64, 0.8, seed=1)
    ptr, _ = O.neighbors(p.xy, p.cutoff)
    cnt = np.diff(ptr).reshape(64, 64)
    interior = cnt[20:44, 20:44]
    expect = math.pi * (p.cutoff / p.h) ** 2
    assert abs(interior.mean() - expect) / expect < 0.02


# ------------------------------------------------------------------ matvec

def test_matvec_cutoff_matches_masked_dense():
    p = W.lattice_problem(40, 0.8, seed=2)
    w = np.random.default_rng(0).standard_normal(p.n)
    y = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    ref = np_matrix(p.xy, p.sigma, p.cutoff) @ w
    assert np.max(np.abs(y - ref)) <= 1e-14 * np.max(np.abs(ref)) * 10
    # other cell sizes give the same truncated operator
    for cf in (0.5, 1.0 / 3.0):
        y2 = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff, c=p.cutoff * cf)
        np.testing.assert_allclose(y2, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_matvec_truncation_error_bound():
    """|A w - A~ w|_inf <= max_i sum_{r_ij > r_c} k(r_ij) |w_j| <= count * exp(-36.98) |w|_inf."""
    p = W.lattice_problem(48, 0.8, seed=3)
    w = np.random.default_rng(1).standard_normal(p.n)
    yc = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    yd = O.matvec_dense(p.xy, w, p.sigma)
    bound = p.n * math.exp(-36.98) * np.abs(w).max()
    assert np.max(np.abs(yc - yd)) <= bound + 1e-15 * np.abs(yd).max()
    np.testing.assert_allclose(yd, np_matrix(p.xy, p.sigma) @ w, rtol=1e-13, atol=1e-13)


def test_matvec_symmetry():
    """A~ is symmetric: e_i^T A~ e_j = e_j^T A~ e_i exactly (same r2 bits)."""
    p = W.lattice_problem(20, 0.8, seed=4)
    a = np.zeros((p.n, p.n))
    for j in range(p.n):
        e = np.zeros(p.n)
        e[j] = 1.0
        a[:, j] = O.matvec_cutoff(p.xy, e, p.sigma, p.cutoff)
    np.testing.assert_array_equal(a, a.T)
    assert np.all(np.linalg.eigvalsh(a) > 0)


def test_normalized_scales_solution():
    """With the 1/(2 pi sigma^2) factor, w scales by 2 pi sigma^2."""
    p = W.lattice_problem(12, 1.0, seed=6)
    w0 = O.dense_solve(p.xy, p.f, p.sigma)
    w1 = O.dense_solve(p.xy, p.f, p.sigma, normalized=True)
    np.testing.assert_allclose(w1, w0 * 2 * math.pi * p.sigma ** 2, rtol=1e-10)


# ---------------------------------------------------------------- Cholesky

def test_cholesky_matches_lapack():
    rng = np.random.default_rng(7)
    m = rng.standard_normal((37, 37))
    a = m @ m.T + 37 * np.eye(37)
    l = O.cholesky(a)
    np.testing.assert_allclose(l, np.linalg.cholesky(a), rtol=1e-12, atol=1e-12)
    b = rng.standard_normal(37)
    np.testing.assert_allclose(O.cholesky_solve(l, b), np.linalg.solve(a, b), rtol=1e-11)


def test_cholesky_rejects_indefinite():
    a = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(O.OracleError):
        O.cholesky(a)


def test_dense_solve_matches_numpy():
    p = W.lattice_problem(20, 0.8, seed=8)
    w = O.dense_solve(p.xy, p.f, p.sigma)
    a = np_matrix(p.xy, p.sigma)
    np.testing.assert_allclose(w, np.linalg.solve(a, p.f), rtol=1e-8, atol=1e-8 * np.abs(w).max())
    # reproduction of f at the nodes
    assert np.linalg.norm(a @ w - p.f) / np.linalg.norm(p.f) < 1e-12


# -------------------------------------------------------------- subdomains

def np_boxes(xy, x0, B, delta):
    """Brute-force geometric box membership (box edges extended to infinity at
    the domain boundary)."""
    xmax, ymax = xy[:, 0].max(), xy[:, 1].max()
    nbx = max(1, int(np.floor((xmax - x0) / B)) + 1)
    nby = max(1, int(np.floor((ymax - x0) / B)) + 1)
    core, ov = [], []
    for by in range(nby):
        for bx in range(nbx):
            def inside(v, k, nb, d):
                lo = -np.inf if k == 0 else x0 + k * B - d
                hi = np.inf if k == nb - 1 else x0 + (k + 1) * B + d
                return (v >= lo) & (v < hi)
            c = inside(xy[:, 0], bx, nbx, 0.0) & inside(xy[:, 1], by, nby, 0.0)
            o = inside(xy[:, 0], bx, nbx, delta) & inside(xy[:, 1], by, nby, delta)
            core.append(np.nonzero(c)[0])
            ov.append(np.nonzero(o)[0])
    return (nbx, nby), core, ov


@pytest.mark.parametrize("n_side,ring", [(64, 1), (37, 1), (30, 2), (16, 0)])
def test_subdomains_match_geometry(n_side, ring):
    p = W.lattice_problem(n_side, 0.8, seed=n_side, ring_points=ring)
    (nbx, nby), cp, ci, op, oi = O.subdomains(p.xy, p.x0, p.x0, p.core_size, p.overlap)
    (rbx, rby), core, ov = np_boxes(p.xy, p.x0, p.core_size, p.overlap)
    assert (nbx, nby) == (rbx, rby)
    for s in range(nbx * nby):
        np.testing.assert_array_equal(ci[cp[s]:cp[s + 1]], core[s])
        np.testing.assert_array_equal(oi[op[s]:op[s + 1]], ov[s])


def test_subdomain_invariants():
    p = W.config_small()
    (nbx, nby), cp, ci, op, oi = O.subdomains(p.xy, p.x0, p.x0, p.core_size, p.overlap)
    assert (nbx, nby) == (16, 16)
    # every point in exactly one core
    np.testing.assert_array_equal(np.sort(ci), np.arange(p.n))
    for s in range(nbx * nby):
        assert set(ci[cp[s]:cp[s + 1]]) <= set(oi[op[s]:op[s + 1]])
    sizes_c = np.diff(cp).reshape(16, 16)
    sizes_o = np.diff(op).reshape(16, 16)
    assert np.all(sizes_c == 16)
    assert np.all(sizes_o[1:-1, 1:-1] == 36)
    assert np.all(sizes_o[0, 1:-1] == 30) and sizes_o[0, 0] == 25


# -------------------------------------------------------------------- RASM

def rasm_dense(p, xy, B, delta):
    """M^{-1} = sum_i ~R_i^T (R_i A~ R_i^T)^{-1} R_i with explicit 0/1 matrices."""
    a = np_matrix(xy, p.sigma, p.cutoff)
    n = xy.shape[0]
    _, core, ov = np_boxes(xy, p.x0, B, delta)
    m = np.zeros((n, n))
    for c, o in zip(core, ov):
        if len(o) == 0:
            continue
        r = np.zeros((len(o), n))
        r[np.arange(len(o)), o] = 1.0
        rt = np.zeros((len(o), n))      # ~R_i: keep rows whose point is in the core
        keep = np.isin(o, c)
        rt[np.arange(len(o))[keep], o[keep]] = 1.0
        ai = r @ a @ r.T
        m += rt.T @ np.linalg.solve(ai, r)
    return m


@pytest.mark.parametrize("ring", [1, 2, 0])
def test_rasm_apply_matches_explicit_matrices(ring):
    p = W.lattice_problem(14, 0.8, seed=21, ring_points=ring)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    v = np.random.default_rng(2).standard_normal(p.n)
    ref = rasm_dense(p, p.xy, p.core_size, p.overlap) @ v
    np.testing.assert_allclose(pr.rasm_apply(v), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_rasm_one_subdomain_is_exact_inverse():
    p = W.lattice_problem(16, 0.8, seed=22)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, -5.0, -5.0, 20.0, 0.0, max_sub_points=4096)
    assert pr.nsub == 1
    v = np.random.default_rng(3).standard_normal(p.n)
    a = np_matrix(p.xy, p.sigma, p.cutoff)
    np.testing.assert_allclose(pr.rasm_apply(v), np.linalg.solve(a, v), rtol=1e-7,
                               atol=1e-7 * np.abs(np.linalg.solve(a, v)).max())
    w, info = pr.solve(p.f)
    assert info.iters == 1 and info.status == 0


def test_rasm_zero_overlap_is_block_jacobi():
    p = W.lattice_problem(12, 0.8, seed=23, ring_points=0)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, 0.0)
    a = np_matrix(p.xy, p.sigma, p.cutoff)
    v = np.random.default_rng(4).standard_normal(p.n)
    cp, ci = pr.core_lists()
    ref = np.zeros(p.n)
    for s in range(pr.nsub):
        idx = ci[cp[s]:cp[s + 1]]
        ref[idx] = np.linalg.solve(a[np.ix_(idx, idx)], v[idx])
    np.testing.assert_allclose(pr.rasm_apply(v), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


# ------------------------------------------------------------------- GMRES

def test_gmres_identity_one_step():
    f = np.random.default_rng(5).standard_normal(50)
    w, info = O.gmres(lambda x: x, None, f)
    assert info.iters == 1
    np.testing.assert_allclose(w, f, rtol=1e-15)


def test_gmres_diagonal_k_distinct_eigenvalues():
    """A diagonal matrix with k distinct values: the Krylov space has dimension k."""
    d = np.repeat([1.0, 2.0, 5.0, 11.0], 25)
    f = np.random.default_rng(6).standard_normal(d.size)
    w, info = O.gmres(lambda x: d * x, None, f, rtol=1e-12)
    assert info.iters <= 4 + 1
    np.testing.assert_allclose(w, f / d, rtol=1e-11)


def test_gmres_full_nonsymmetric_exact_in_n_steps():
    rng = np.random.default_rng(7)
    n = 24
    a = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    f = rng.standard_normal(n)
    w, info = O.gmres(lambda x: a @ x, None, f, m=n, rtol=1e-13)
    assert info.iters <= n and info.restarts == 1
    np.testing.assert_allclose(w, np.linalg.solve(a, f), rtol=1e-10)
    # GMRES minimises the residual over the growing Krylov space: monotone
    assert np.all(np.diff(info.history) <= 1e-15)


def test_gmres_right_preconditioned_matches_solve():
    rng = np.random.default_rng(8)
    n = 60
    a = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.3
    dinv = 1.0 / np.diag(a)
    f = rng.standard_normal(n)
    w, info = O.gmres(lambda x: a @ x, lambda x: dinv * x, f, m=10, rtol=1e-13, max_iters=500)
    assert info.status == 0 and info.restarts >= 2
    np.testing.assert_allclose(w, np.linalg.solve(a, f), rtol=1e-10)
    assert np.linalg.norm(f - a @ w) / np.linalg.norm(f) <= 1e-13


# -------------------------------------------------------------- end to end

def test_small_solve_reaches_tolerance_and_matches_dense():
    p = W.config_small()
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    w, info = pr.solve(p.f, m=30, rtol=1e-13)
    assert info.status == 0 and info.relres <= 1e-13
    a = np_matrix(p.xy, p.sigma, p.cutoff)
    assert np.linalg.norm(p.f - a @ w) / np.linalg.norm(p.f) <= 1.5e-13
    # the truncated and the untruncated systems have nearly the same solution
    wd = O.dense_solve(p.xy, p.f, p.sigma)
    assert np.linalg.norm(w - wd) / np.linalg.norm(wd) < 1e-6


def test_paper_point_counts():
    """N = (1/h + 1)^2 on [0, 1]^2 reproduces every N the paper prints."""
    with open(os.path.join(GOLDEN, "paper_point_counts.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        p = W.unit_square_problem(c["h_over_sigma"], sigma=c["sigma"]) if c["N"] < 10 ** 6 else None
        if p is not None:
            assert p.n == c["N"], c
        h = c["h_over_sigma"] * c["sigma"] if "sigma" in c else None
        if h:
            assert (int(round(1.0 / h)) + 1) ** 2 == c["N"]
    assert 7112 ** 2 == 50580544


@pytest.mark.slow
def test_iterations_independent_of_n():
    """Sec. 3.2: fixed h/sigma, B/sigma, D/sigma give the same iteration count
    as N grows (allow +-2 for rounding)."""
    its = []
    for n_side in (48, 96):
        p = W.lattice_problem(n_side, 1.0, seed=3)
        pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
        _, info = pr.solve(p.f)
        assert info.status == 0
        its.append(info.iters)
    assert abs(its[0] - its[1]) <= 2, its


@pytest.mark.slow
def test_paper_parameters_converge_quickly():
    """Sec. 3.2: with B = 5 sigma, D = 1.9 B on a lattice and h/sigma >= 0.9, the
    method converges in fewer than 20 iterations (Franke's function)."""
    p = W.unit_square_problem(1.0, sigma=0.01)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    _, info = pr.solve(p.f, rtol=1e-13)
    assert info.status == 0
    assert info.iters < 20, info.iters


# ------------------------------------------------- ASM and evaluation

def asm_dense(p, B, delta):
    """sum_i R_i^T A_i^{-1} R_i (Eq. asm) from explicit numpy matrices."""
    a = np_matrix(p.xy, p.sigma, p.cutoff)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, B, delta)
    op, oi = pr.overlap_lists()
    m = np.zeros((p.n, p.n))
    for s in range(pr.nsub):
        o = oi[op[s]:op[s + 1]]
        m[np.ix_(o, o)] += np.linalg.inv(a[np.ix_(o, o)])
    return m


@pytest.mark.parametrize("ring", [1, 2])
def test_asm_apply_matches_explicit_matrices(ring):
    p = W.lattice_problem(14, 0.8, seed=31, ring_points=ring)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap, additive=True)
    v = np.random.default_rng(5).standard_normal(p.n)
    ref = asm_dense(p, p.core_size, p.overlap) @ v
    np.testing.assert_allclose(pr.rasm_apply(v), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_asm_is_symmetric_and_reduces_to_block_jacobi():
    p = W.lattice_problem(12, 0.8, seed=32)
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap, additive=True)
    rng = np.random.default_rng(6)
    u, v = rng.standard_normal(p.n), rng.standard_normal(p.n)
    a, b = v @ pr.rasm_apply(u), u @ pr.rasm_apply(v)
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))      # M^-1 of Eq. asm is symmetric (Eq. rasm's is not)
    q = W.lattice_problem(12, 0.8, seed=33, ring_points=0)
    r0 = O.Problem(q.xy, q.sigma, q.cutoff, q.x0, q.x0, q.core_size, 0.0)
    a0 = O.Problem(q.xy, q.sigma, q.cutoff, q.x0, q.x0, q.core_size, 0.0, additive=True)
    np.testing.assert_array_equal(a0.rasm_apply(u[:q.n]), r0.rasm_apply(u[:q.n]))   # no overlap: identical


def test_rasm_converges_faster_than_asm():
    """Sec. 2.2: the restricted variant converges in fewer GMRES steps than the
    plain additive one on the same subdomains (paper sizes B = 5 sigma, D = 1.9 B)."""
    p = W.unit_square_problem(0.9, sigma=0.02, seed=34)
    it = {}
    for additive in (False, True):
        pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap, additive=additive)
        _, info = pr.solve(p.f, max_iters=600)
        assert info.status == 0
        it[additive] = info.iters
    assert it[False] < it[True], it


def test_eval_matches_numpy_definition():
    p = W.lattice_problem(24, 0.8, seed=35)
    rng = np.random.default_rng(7)
    w = rng.standard_normal(p.n)
    xe = rng.uniform(-1.1, 1.1, (3000, 2))
    dx = xe[:, None, 0] - p.xy[None, :, 0]
    dy = xe[:, None, 1] - p.xy[None, :, 1]
    r2 = dx * dx + dy * dy
    k = np.exp(-r2 / (2 * p.sigma * p.sigma))
    k[r2 > p.cutoff * p.cutoff] = 0.0
    ref = k @ w
    got = O.eval_points(p.xy, w, xe, p.sigma, p.cutoff)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    # at the centres the interpolant is the matvec (same truncated operator)
    np.testing.assert_allclose(O.eval_points(p.xy, w, p.xy, p.sigma, p.cutoff),
                               O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff), rtol=0, atol=1e-14 * np.abs(ref).max())


def test_eval_single_centre_and_far_points():
    xy = np.array([[0.3, -0.2]])
    sigma, rc = 0.05, 0.43
    xe = np.array([[0.3, -0.2], [0.35, -0.2], [0.3, 0.0], [5.0, 5.0], [0.3 + 0.43, -0.2], [0.3 + 0.4301, -0.2]])
    got = O.eval_points(xy, np.array([2.5]), xe, sigma, rc)
    r2 = ((xe - xy) ** 2).sum(1)
    ref = 2.5 * np.exp(-r2 / (2 * sigma * sigma))
    ref[r2 > rc * rc] = 0.0
    np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)
    assert got[3] == 0.0 and got[5] == 0.0 and got[4] > 0.0
