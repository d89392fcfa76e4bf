"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Index work (binning, neighbour and subdomain lists) must match bit for bit.
FP64 matvec: relative error <= 1e-13 (each entry is one exp plus an FMA chain;
the two sides differ only in rounding order and in the exp implementation).
Solves: the true relative residual, recomputed by the oracle's own FP64
matvec, must be <= 1e-13.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_5413_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rbf():
    from paper_0909_5413_gb300 import rbf as R
    R.load()
    return R


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make_ctx(rbf, xy, sigma, rc, cell=0.0, normalized=False, sym64=False):
    ctx = rbf.Context(0)
    if sym64:   # the symmetric FP64 matvec (chosen at binning)
        rbf.rbf_set_option(ctx.handle, rbf.RBF_OPT_SYMMETRIC_F64, 1)
    xyd = dev(xy)
    rbf.rbf_bin(ctx.handle, xyd, xy.shape[0], rbf.RbfParams(sigma, rc, cell, int(normalized)))
    return ctx, xyd


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_points(n, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(lo, hi, size=(n, 2)))


# ------------------------------------------------------------------ binning

def bin_cases():
    p = W.config_small()
    yield "lattice64", p.xy, p.sigma, p.cutoff, 0.0
    yield "lattice64_half_cells", p.xy, p.sigma, p.cutoff, p.cutoff / 2
    q = W.lattice_problem(37, 0.8, seed=37)
    yield "lattice37_ragged", q.xy, q.sigma, q.cutoff, 0.0
    for n in (1, 2, 15, 16, 17, 255):
        yield f"rand{n}", random_points(n, n), 0.05, 0.3, 0.0
    yield "one_cell", random_points(300, 9, 0.0, 0.01), 0.001, 1.0, 0.0
    a, b = random_points(100, 11, -1.0, -0.5), random_points(100, 12, 0.5, 1.0)
    yield "gap", np.ascontiguousarray(np.vstack([a, b])), 0.02, 0.2, 0.0
    e = np.array([[0.0, 0.0], [0.25, 0.0], [0.5, 0.5], [0.25, 0.0], [0.75, 1.0], [1.0, 1.0]])
    yield "edges_duplicates", e, 0.05, 0.25, 0.0


@pytest.mark.parametrize("case", list(bin_cases()), ids=[c[0] for c in bin_cases()])
def test_binning_bit_exact(rbf, case):
    name, xy, sigma, rc, cell = case
    ctx, _ = make_ctx(rbf, xy, sigma, rc, cell)
    g, perm, cs = O.bin_points(xy, cell if cell > 0 else rc)
    ncx, ncy, bbox = rbf.rbf_get_grid(ctx.handle)
    assert (ncx, ncy) == (g.ncx, g.ncy)
    assert bbox == (g.xmin, g.ymin, g.xmax, g.ymax)
    pd = torch.empty(xy.shape[0], dtype=torch.int32, device="cuda")
    cd = torch.empty(ncx * ncy + 1, dtype=torch.int32, device="cuda")
    rbf.rbf_get_bins(ctx.handle, pd, cd)
    np.testing.assert_array_equal(host(pd), perm)
    np.testing.assert_array_equal(host(cd), cs)
    ctx.close()


def test_binning_bit_exact_1m(rbf):
    p = W.config_1m()
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    g, perm, cs = O.bin_points(p.xy, p.cutoff)
    ncx, ncy, _ = rbf.rbf_get_grid(ctx.handle)
    pd = torch.empty(p.n, dtype=torch.int32, device="cuda")
    cd = torch.empty(ncx * ncy + 1, dtype=torch.int32, device="cuda")
    rbf.rbf_get_bins(ctx.handle, pd, cd)
    np.testing.assert_array_equal(host(pd), perm)
    np.testing.assert_array_equal(host(cd), cs)
    ctx.close()


# --------------------------------------------------------------- neighbours

@pytest.mark.parametrize("n_side,cfac", [(40, 1.0), (64, 1.0), (33, 0.5), (21, 1.0 / 3.0)])
def test_neighbor_lists_bit_exact(rbf, n_side, cfac):
    p = W.lattice_problem(n_side, 0.8, seed=n_side)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff, p.cutoff * cfac)
    total = rbf.rbf_count_neighbors(ctx.handle)
    ptr = torch.empty(p.n + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(total, dtype=torch.int32, device="cuda")
    rbf.rbf_get_neighbors(ctx.handle, ptr, idx, total)
    rptr, ridx = O.neighbors(p.xy, p.cutoff, c=p.cutoff * cfac)
    np.testing.assert_array_equal(host(ptr), rptr)
    np.testing.assert_array_equal(host(idx), ridx)
    ctx.close()


def test_neighbor_capacity_error(rbf):
    p = W.lattice_problem(16, 0.8, seed=1)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    total = rbf.rbf_count_neighbors(ctx.handle)
    ptr = torch.empty(p.n + 1, dtype=torch.int64, device="cuda")
    idx = torch.empty(total, dtype=torch.int32, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_get_neighbors(ctx.handle, ptr, idx, total - 1)
    assert e.value.status == 1
    ctx.close()


# ------------------------------------------------------------ subdomains

def sub_cases():
    yield "lattice64", W.config_small()
    yield "lattice37", W.lattice_problem(37, 0.8, seed=3)
    yield "ring2", W.lattice_problem(30, 0.8, seed=4, ring_points=2)
    yield "ring0", W.lattice_problem(16, 0.8, seed=5, ring_points=0)
    yield "unit_square_paper", W.unit_square_problem(1.0, sigma=0.02)


def gpu_subdomains(rbf, ctx):
    nbx, nby, ct, ot = rbf.rbf_get_subdomain_sizes(ctx.handle)
    ns = nbx * nby
    cp = torch.empty(ns + 1, dtype=torch.int32, device="cuda")
    op = torch.empty(ns + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(max(ct, 1), dtype=torch.int32, device="cuda")
    oi = torch.empty(max(ot, 1), dtype=torch.int32, device="cuda")
    rbf.rbf_get_subdomains(ctx.handle, cp, ci, op, oi)
    return (nbx, nby), host(cp), host(ci)[:ct], host(op), host(oi)[:ot]


@pytest.mark.parametrize("case", list(sub_cases()), ids=[c[0] for c in sub_cases()])
def test_subdomain_lists_bit_exact(rbf, case):
    _, p = case
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 0, 0))
    (nbx, nby), cp, ci, op, oi = gpu_subdomains(rbf, ctx)
    (rbx, rby), rcp, rci, rop, roi = O.subdomains(p.xy, p.x0, p.x0, p.core_size, p.overlap)
    assert (nbx, nby) == (rbx, rby)
    np.testing.assert_array_equal(cp, rcp)
    np.testing.assert_array_equal(ci, rci)
    np.testing.assert_array_equal(op, rop)
    np.testing.assert_array_equal(oi, roi)
    ctx.close()


def test_subdomain_lists_bit_exact_1m(rbf):
    p = W.config_1m()
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 64, 0))
    (nbx, nby), cp, ci, op, oi = gpu_subdomains(rbf, ctx)
    (rbx, rby), rcp, rci, rop, roi = O.subdomains(p.xy, p.x0, p.x0, p.core_size, p.overlap)
    assert (nbx, nby) == (rbx, rby) == (256, 256)
    np.testing.assert_array_equal(cp, rcp)
    np.testing.assert_array_equal(ci, rci)
    np.testing.assert_array_equal(op, rop)
    np.testing.assert_array_equal(oi, roi)
    ctx.close()


def test_subdomain_too_large_is_reported(rbf):
    p = W.lattice_problem(32, 0.8, seed=6)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, 8 * p.h, p.h, 64, 0))
    assert e.value.status == 5
    # the default cap is the largest supported list, 192 points: 14 x 14 boxes exceed it
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, 12 * p.h, p.h, 0, 0))
    assert e.value.status == 5
    # 12 x 12 = 144 points (the paper's D = 1.9 B at h/sigma = 0.8) fit
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, 10 * p.h, p.h, 0, 0))
    ctx.close()


def test_duplicate_points_not_spd(rbf):
    p = W.lattice_problem(12, 0.8, seed=7)
    xy = p.xy.copy()
    xy[5] = xy[4]
    ctx, _ = make_ctx(rbf, xy, p.sigma, p.cutoff)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 64, 0))
    assert e.value.status == 4
    ctx.close()


def test_state_errors(rbf):
    p = W.lattice_problem(8, 0.8, seed=8)
    ctx = rbf.Context(0)
    v = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_matvec(ctx.handle, v, v)
    assert e.value.status == 8
    rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_rasm_apply(ctx.handle, v, v)
    assert e.value.status == 8
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(-1.0, p.cutoff, 0.0, 0))
    assert e.value.status == 1
    ctx.close()


# --------------------------------------------------------------------- exp

@pytest.mark.parametrize("variant", [0, 2])
def test_library_exp_against_cuda_exp(rbf, variant):
    """The table-driven exps (Tang's method, 64 and 2048 entries) agree with
    CUDA's exp() to a few ulp plus t ulp: the 2048-entry variant folds the
    rounded constant 2048/ln 2 into its argument, an error of t * eps relative
    (below 1e-14 for t <= 37, the cutoff range; the same order as rounding the
    constant 1/(2 sigma^2) itself)."""
    ctx = rbf.Context(0)
    rng = np.random.default_rng(variant)
    t = np.concatenate([rng.uniform(0.0, 40.0, 200000), rng.uniform(0.0, 670.0, 50000),
                        np.array([0.0, 1e-300, 1e-12, 0.5, 36.98, 100.0, 669.9]),
                        np.arange(0, 40, 1.0 / 64)])
    td = dev(t)
    a = torch.empty_like(td)
    b = torch.empty_like(td)
    rbf.rbf_debug_exp(ctx.handle, td, a, variant)
    rbf.rbf_debug_exp(ctx.handle, td, b, 1)
    got, ref = host(a), host(b)
    rel = np.abs(got - ref) / ref
    bound = 4 * 2.0 ** -52 + t * 2.0 ** -52
    assert np.all(rel <= bound), (rel.max(), t[(rel / bound).argmax()])
    inside = t <= 37.0
    assert rel[inside].max() <= 1e-14
    ctx.close()


@pytest.mark.parametrize("case", ["lattice64", "lattice1024_scale", "offset_domain", "wide_cutoff"])
def test_fixed_point_kernel_values(rbf, case):
    """The FP64 matvec's kernel value (64-bit fixed-point offsets and exp, FP64
    bits assembled at the end) against exp(-r2 s) evaluated in long double
    from the same FP64 coordinates and the same FP64 s = 1/(2 sigma^2): within
    4e-16 relative over the whole cutoff disc for r_c = 8.6 sigma, 0 beyond it.
    The log2 argument carries about 57 - log2(t_max) fraction bits, so at
    r_c = 30 sigma (t up to 450) the bound is 2e-15 -- still below the FP64
    rounding of the argument itself there (t 2^-53 = 5e-14)."""
    rng = np.random.default_rng(17)
    if case == "lattice64":
        p = W.config_small()
        xy, sigma, rc = p.xy, p.sigma, p.cutoff
    elif case == "lattice1024_scale":   # sigma and r_c of the 1M-point lattice, on a small point set
        sigma = (2.0 / 1023) / 0.8
        rc = 8.6 * sigma
        xy = rng.uniform(-1.0, 1.0, (4096, 2))
    elif case == "offset_domain":       # coordinates far from the origin (few low bits left)
        sigma, rc = 0.01, 0.086
        xy = 1000.0 + rng.uniform(0.0, 1.0, (4096, 2))
    else:                               # r_c = 30 sigma: longer exp range (t up to 450)
        sigma = 0.02
        rc = 30 * sigma
        xy = rng.uniform(-1.0, 1.0, (4096, 2))
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, dev(xy), xy.shape[0], rbf.RbfParams(sigma, rc, 0.0, 0))
    m = 200000
    i = rng.integers(0, xy.shape[0], m)
    r = rc * np.sqrt(rng.uniform(0.0, 1.0, m))
    r[:64] = rc * (1.0 - np.logspace(-15, -1, 64))   # at the cutoff
    r[64:96] = 0.0
    th = rng.uniform(0.0, 2.0 * np.pi, m)
    xj = xy[i, 0] + r * np.cos(th)
    yj = xy[i, 1] + r * np.sin(th)
    pairs = np.stack([xy[i, 0], xy[i, 1], xj, yj], axis=1)
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    rbf.rbf_debug_kernel_pairs(ctx.handle, dev(pairs), out)
    got = host(out)
    ctx.close()
    L = np.longdouble
    dx = pairs[:, 0].astype(L) - pairs[:, 2].astype(L)
    dy = pairs[:, 1].astype(L) - pairs[:, 3].astype(L)
    s = L(1.0 / (2.0 * sigma * sigma))
    ref = np.exp(-(dx * dx + dy * dy) * s)
    ex = pairs[:, 0] - pairs[:, 2]
    ey = pairs[:, 1] - pairs[:, 3]
    inside = (ex * ex + ey * ey) <= rc * rc   # the FP64 test of the index-list definition
    assert np.all(got[~inside] == 0.0)
    rel = np.abs(got[inside].astype(L) - ref[inside]) / ref[inside]
    bound = 2e-15 if case == "wide_cutoff" else 4e-16
    assert float(rel.max()) <= bound, float(rel.max())


def test_bin_rejects_cutoff_below_fixed_point_resolution(rbf):
    xy = 1.0e12 + np.random.default_rng(1).uniform(0.0, 1.0, (100, 2))
    ctx = rbf.Context(0)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_bin(ctx.handle, dev(xy), 100, rbf.RbfParams(1e-4, 8.6e-4, 0.0, 0))
    assert e.value.status == 1
    ctx.close()


# ------------------------------------------------------------------ matvec

def matvec_cases():
    yield "lattice64", W.config_small(), 0.0, False
    yield "lattice64_normalized", W.config_small(), 0.0, True
    yield "lattice37_half_cells", W.lattice_problem(37, 0.8, seed=9), 0.5, False
    yield "lattice50_ratio1", W.lattice_problem(50, 1.0, seed=10), 1.0 / 3.0, False
    yield "lattice3", W.lattice_problem(3, 0.8, seed=11), 0.0, False


@pytest.mark.parametrize("case", list(matvec_cases()), ids=[c[0] for c in matvec_cases()])
def test_matvec_f64_matches_oracle(rbf, case):
    _, p, cf, normalized = case
    cell = p.cutoff * cf if cf > 0 else 0.0
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff, cell, normalized)
    w = np.random.default_rng(1).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y, rbf.RBF_FP64)
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff, normalized=normalized)
    got = host(y)
    assert rel_err(got, ref) <= 1e-13
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    ctx.close()


def test_matvec_f64_matches_oracle_1m(rbf):
    p = W.config_1m()
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    w = np.random.default_rng(2).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y, rbf.RBF_FP64)
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    got = host(y)
    assert rel_err(got, ref) <= 1e-13
    # element by element: every entry within 1e-13 of the largest
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    ctx.close()


def test_matvec_dense_limit(rbf):
    """A cutoff beyond the domain gives the untruncated dense product."""
    p = W.lattice_problem(20, 1.0, seed=12)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, 10.0)
    w = np.random.default_rng(3).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y)
    assert rel_err(host(y), O.matvec_dense(p.xy, w, p.sigma)) <= 1e-13
    ctx.close()


def test_matvec_f32_error(rbf):
    """FP32 matvec on cell-local coordinates: relative error ~1e-6 (FP32 rounding of
    the scaled offsets, |dX|^2 up to 53 in exp2 units, and ex2.approx)."""
    p = W.config_small()
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    w = np.random.default_rng(4).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y, rbf.RBF_FP32)
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    assert rel_err(host(y), ref) <= 2e-5
    ctx.close()


# ------------------------------------------------------------------- RASM

# The GPU applies stored rows of A_i^{-1} while the oracle solves with the
# Cholesky factor; both are backward stable, so they differ by about
# cond(A_i) * eps. cond(A_i) for the 6 x 6-point boxes at h/sigma = 0.8 is
# about 1e4, so 1e-10 leaves a wide margin; the wider ring needs more.
@pytest.mark.parametrize("ring,tol", [(1, 1e-10), (2, 1e-8), (0, 1e-10)])
def test_rasm_apply_matches_oracle(rbf, ring, tol):
    p = W.lattice_problem(40, 0.8, seed=13, ring_points=ring)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 64, 0))
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    v = np.random.default_rng(5).standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_rasm_apply(ctx.handle, dev(v), z)
    got, ref = host(z), pr.rasm_apply(v)
    assert rel_err(got, ref) <= tol
    # element by element: a wrong core write in one subdomain cannot hide under the norm
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    ctx.close()


# FP32 inverses: computed in FP64 and rounded (precision 2), the FP32 rounding
# of W_i alone; computed in FP32 on the tensor cores (precision 1), whose block
# sweep leaves about cond(A_i) * 2^-23 (cond about 2e4 at h/sigma = 0.8).
@pytest.mark.parametrize("precision,tol", [(2, 1e-5), (1, 3e-3)])
def test_rasm_apply_f32_factors(rbf, precision, tol):
    p = W.config_small()
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff)
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 64, precision))
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    v = np.random.default_rng(6).standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_rasm_apply(ctx.handle, dev(v), z)
    got, ref = host(z), pr.rasm_apply(v)
    assert rel_err(got, ref) <= tol
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    ctx.close()


# ------------------------------------------------------------------- solve

def solve_gpu(rbf, p, mixed=False, w0=None, **kw):
    cfg = rbf.config_for(p, mixed=mixed, **kw)
    ctx = rbf.Context(0)
    xyd = dev(p.xy)
    ctx.bin(xyd, cfg)
    ctx.rasm_setup(cfg)
    w = dev(np.zeros(p.n) if w0 is None else w0)
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    out = host(w)
    ctx.close()
    return st, info, out


def oracle_relres(p, w):
    r = p.f - O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    return float(np.linalg.norm(r) / np.linalg.norm(p.f))


def test_solve_f64_small_matches_oracle(rbf):
    p = W.config_small()
    st, info, w = solve_gpu(rbf, p)
    assert st == 0
    assert info.relres <= 1e-13
    assert oracle_relres(p, w) <= 1e-13
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    wo, oinfo = pr.solve(p.f)
    # both solve the same SPD system to 1e-13: |dw|/|w| <= cond(A~) * 2e-13
    assert rel_err(w, wo) <= 1e-6
    assert abs(info.iters - oinfo.iters) <= 3, (info.iters, oinfo.iters)
    # and the dense direct solve of the untruncated system
    wd = O.dense_solve(p.xy, p.f, p.sigma)
    assert rel_err(w, wd) <= 1e-6


def test_solve_f64_1m_reaches_tolerance(rbf):
    p = W.config_1m()
    st, info, w = solve_gpu(rbf, p)
    assert st == 0 and info.relres <= 1e-13
    assert oracle_relres(p, w) <= 1e-13


def test_solve_mixed_small(rbf):
    p = W.config_small()
    st, info, w = solve_gpu(rbf, p, mixed=True)
    assert st == 0, info.as_dict()
    assert info.refinements >= 1
    assert oracle_relres(p, w) <= 1e-13


def test_solve_mixed_1m(rbf):
    p = W.config_1m()
    st, info, w = solve_gpu(rbf, p, mixed=True)
    assert st == 0, info.as_dict()
    assert oracle_relres(p, w) <= 1e-13


@pytest.mark.slow
def test_solve_mixed_51m_reaches_tolerance(rbf):
    """The 7168 x 7168 lattice (N = 51,380,224) with FP32 inner solves: the true
    relative residual, recomputed by the oracle's FP64 matvec on the host, is
    <= 1e-13."""
    p = W.config_51m()
    st, info, w = solve_gpu(rbf, p, mixed=True, factor_precision=rbf.RBF_FP32)
    assert st == 0, info.as_dict()
    assert oracle_relres(p, w) <= 1e-13


def test_solve_edge_single_point(rbf):
    p = W.lattice_problem(1, 0.8, seed=1)
    xy = np.array([[0.3, -0.2]])
    from dataclasses import replace
    q = replace(p, xy=xy, f=np.array([2.5]), sigma=0.1, cutoff=0.86, x0=-1.0, core_size=0.5, overlap=0.1)
    st, info, w = solve_gpu(rbf, q)
    assert st == 0
    np.testing.assert_allclose(w, [2.5], rtol=1e-15)


def test_solve_zero_rhs(rbf):
    from dataclasses import replace
    p = W.lattice_problem(10, 0.8, seed=2)
    q = replace(p, f=np.zeros(p.n))
    st, info, w = solve_gpu(rbf, q, w0=np.ones(p.n))
    assert st == 0 and np.all(w == 0.0)


def test_solve_warm_start_resumes(rbf):
    """A solve stopped early returns its w; a second call continues from it."""
    p = W.lattice_problem(48, 0.8, seed=3)
    st, info, w1 = solve_gpu(rbf, p, max_iters=20)
    assert st == 6 and info.iters == 20
    st2, info2, w2 = solve_gpu(rbf, p, w0=w1)
    assert st2 == 0 and oracle_relres(p, w2) <= 1e-13


def test_interpolate_host_matches_device_path(rbf):
    p = W.config_small()
    cfg = rbf.config_for(p)
    xy_h = torch.from_numpy(p.xy.copy()).pin_memory()
    f_h = torch.from_numpy(p.f.copy()).pin_memory()
    w_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    ctx = rbf.Context(0)
    st, info = ctx.interpolate_host(xy_h, f_h, w_h, cfg)
    assert st == 0
    _, _, w = solve_gpu(rbf, p)
    np.testing.assert_array_equal(w_h.numpy(), w)
    assert ctx.launches > 0
    # a second call of the same size reuses the context's device copies: no
    # allocation, the same bits; a smaller problem then fits in them
    held = rbf.rbf_device_bytes(ctx.handle)
    w_h.zero_()
    st, info = ctx.interpolate_host(xy_h, f_h, w_h, cfg)
    assert st == 0 and rbf.rbf_device_bytes(ctx.handle) == held
    np.testing.assert_array_equal(w_h.numpy(), w)
    q = W.lattice_problem(40, 0.85, seed=9)
    wq = torch.zeros(q.n, dtype=torch.float64).pin_memory()
    st, info = ctx.interpolate_host(torch.from_numpy(q.xy.copy()).pin_memory(),
                                    torch.from_numpy(q.f.copy()).pin_memory(), wq, rbf.config_for(q))
    assert st == 0 and oracle_relres(q, wq.numpy()) <= 1e-13
    ctx.close()


# ------------------------------------------------- tiles, cell sizes, tuner

def matvec_with(rbf, p, w, cell, t64, t32):
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, cell, 0, t64, t32))
    y64 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    y32 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y64, rbf.RBF_FP64)
    rbf.rbf_matvec(ctx.handle, dev(w), y32, rbf.RBF_FP32)
    out = host(y64), host(y32)
    ctx.close()
    return out


@pytest.mark.parametrize("cf", [1.0, 0.5, 1.0 / 3.0])
def test_matvec_tiles_and_cell_sizes(rbf, cf):
    """Every tile gives the same bits (the per-target summation order does not
    depend on it); every cell size gives the oracle's truncated product."""
    p = W.lattice_problem(72, 0.8, seed=61)
    w = np.random.default_rng(12).standard_normal(p.n)
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    res = {t: matvec_with(rbf, p, w, cf * p.cutoff, t, t) for t in (32, 64, 128)}
    for t in (32, 64):
        np.testing.assert_array_equal(res[t][0], res[128][0])
        np.testing.assert_array_equal(res[t][1], res[128][1])
    assert rel_err(res[128][0], ref) <= 1e-13
    assert rel_err(res[128][1], ref) <= 2e-5


def test_tile_validation(rbf):
    p = W.lattice_problem(12, 0.8, seed=62)
    ctx = rbf.Context(0)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0, 48, 0))
    assert e.value.status == 1
    ctx.close()


@pytest.mark.parametrize("w32", [0.0, 26.0])
def test_tune_picks_a_valid_setting_and_solves(rbf, w32):
    p = W.lattice_problem(160, 0.8, seed=63)
    ctx = rbf.Context(0)
    xyd = dev(p.xy)
    best, score = rbf.rbf_tune(ctx.handle, xyd, p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0), 1.0, w32)
    assert best.tile_f64 in (32, 64, 128) and best.tile_f32 in (32, 64, 128)
    assert any(abs(best.cell_size - f * p.cutoff) <= 1e-12 * p.cutoff for f in (1.0, 0.5, 1.0 / 3.0))
    assert score > 0.0
    # the context is binned with the pick: the matvec is the oracle's, and a solve converges
    w = np.random.default_rng(13).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y)
    assert rel_err(host(y), O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)) <= 1e-13
    mixed = w32 > 0
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, 0, int(mixed)))
    wd = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = rbf.rbf_solve(ctx.handle, dev(p.f), wd, rbf.RbfSolveParams(1e-13, 30, 5000, int(mixed), 60, 1e-5),
                             check=False)
    assert st == 0 and info.relres <= 1e-13
    ctx.close()


# ------------------------------------------------- symmetric FP64 matvec

@pytest.mark.parametrize("n_side,ratio,normalized", [(96, 0.8, False), (61, 0.9, True), (80, 1.0, False),
                                                     (40, 0.85, False)])
def test_symmetric_f64_matvec(rbf, n_side, ratio, normalized):
    """Each neighbouring pair of cells once (kernel values shared by both
    directions, column sums gathered in a fixed order) against the stencil
    kernel and the oracle, element by element; and the same bits on a second call."""
    p = W.lattice_problem(n_side, ratio, seed=600 + n_side)
    ctx, _ = make_ctx(rbf, p.xy, p.sigma, p.cutoff, 0.0, normalized, sym64=True)
    w = np.random.default_rng(7).standard_normal(p.n)
    ys, yt, y2 = (torch.empty(p.n, dtype=torch.float64, device="cuda") for _ in range(3))
    rbf.rbf_matvec(ctx.handle, dev(w), ys)
    rbf.rbf_matvec(ctx.handle, dev(w), y2)
    rbf.rbf_set_option(ctx.handle, rbf.RBF_OPT_SYMMETRIC_F64, 0)
    rbf.rbf_matvec(ctx.handle, dev(w), yt)
    a, b, c = host(ys), host(yt), host(y2)
    np.testing.assert_array_equal(a, c)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff, normalized=normalized)
    assert np.max(np.abs(a - ref)) <= 1e-13 * np.max(np.abs(ref))
    ctx.close()


def test_symmetric_f64_matvec_uneven_points(rbf):
    """Uniform random points (empty and crowded cells, ragged edges)."""
    rng = np.random.default_rng(12)
    xy = np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(9000, 2)))
    sigma, rc = 0.015, 0.129
    ctx, _ = make_ctx(rbf, xy, sigma, rc, sym64=True)
    w = rng.standard_normal(xy.shape[0])
    y = torch.empty(xy.shape[0], dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y)
    ref = O.matvec_cutoff(xy, w, sigma, rc)
    got = host(y)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    ctx.close()
