"""The mixed form with a shorter inner cutoff: the FP32 inner solves run on a
second grid (cells of r_i = 6.1 sigma, its own order, subdomain lists
re-indexed), the FP64 residual keeps r_c. The solves must still reach the
true relative residual 1e-13 of the r_c system, a problem must give the same
bits alone and in a batch, and the context's other operators must not change."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def single(rbf, p, ri, **kw):
    cfg = rbf.config_for(p, mixed=True, factor_precision=rbf.RBF_FP32, inner_cutoff=ri, **kw)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    out = host(w)
    return ctx, st, info, out


@pytest.mark.parametrize("n_side,ratio", [(96, 0.8), (160, 0.9), (64, 1.0)])
def test_inner_grid_solve_reaches_tolerance(rbf, n_side, ratio):
    p = W.lattice_problem(n_side, ratio, seed=70 + n_side)
    ctx, st, info, w = single(rbf, p, 6.1)
    assert st == 0 and info.relres <= 1e-13, info.as_dict()
    r = p.f - O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13
    _, st0, info0, _ = single(rbf, p, 0.0)
    assert st0 == 0
    assert info.iters <= 1.5 * info0.iters + 30, (info.iters, info0.iters)
    ctx.close()


def test_inner_grid_leaves_other_operators_alone(rbf):
    p = W.lattice_problem(80, 0.85, seed=71)
    cfg = rbf.config_for(p, mixed=True, factor_precision=rbf.RBF_FP32, inner_cutoff=6.1)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    v = dev(np.random.default_rng(3).standard_normal(p.n))
    before = []
    for prec in (0, 1):
        y = torch.empty(p.n, dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(ctx.handle, v, y, prec)
        before.append(host(y))
    z0 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_rasm_apply(ctx.handle, v, z0)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg)
    for prec in (0, 1):
        y = torch.empty(p.n, dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(ctx.handle, v, y, prec)
        np.testing.assert_array_equal(host(y), before[prec])
    z1 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_rasm_apply(ctx.handle, v, z1)
    np.testing.assert_array_equal(host(z1), host(z0))
    ctx.close()


def batch_solve(rbf, probs):
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP32)
    ctx = rbf.Context(0)
    rbf.rbf_bin_batch(ctx.handle, dev(xy), ptr, params)
    rbf.rbf_rasm_setup_batch(ctx.handle, rasm)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    sp = rbf.RbfSolveParams(1e-13, 30, 5000, 1, 200, 1e-5, 6.1)
    st, infos = rbf.rbf_solve_batch(ctx.handle, dev(f), w, sp, len(probs), check=False)
    out = host(w)
    ctx.close()
    return st, infos, out, ptr


def test_inner_grid_batch_alone_equals_mix(rbf):
    """In a batch, each problem's inner grid and order are its own: the same
    bits alone and in the mix; every problem reaches the tolerance."""
    probs = [W.lattice_problem(n, r, seed=80 + n, rhs="four_gaussians") for n, r in ((40, 0.9), (72, 0.8), (24, 1.0))]
    st, infos, wb, ptr = batch_solve(rbf, probs)
    assert st == 0, [i.as_dict() for i in infos]
    for b, p in enumerate(probs):
        r = p.f - O.matvec_cutoff(p.xy, wb[ptr[b]:ptr[b + 1]], p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13
        st1, _, w1, _ = batch_solve(rbf, [p])
        assert st1 == 0
        np.testing.assert_array_equal(w1, wb[ptr[b]:ptr[b + 1]])


def host_candidates(xy, c):
    """Sum over the cells of side c (origin at the bounding box's low corner,
    the last cell clamped) of points x points of the 3 x 3 stencil."""
    lo, hi = xy.min(axis=0), xy.max(axis=0)
    nc = (np.floor((hi - lo) / c) + 1).astype(np.int64)
    cell = np.minimum(np.floor((xy - lo) / c).astype(np.int64), nc - 1)
    cnt = np.zeros((nc[1], nc[0]), dtype=np.int64)
    np.add.at(cnt, (cell[:, 1], cell[:, 0]), 1)
    pad = np.pad(cnt, 1)
    win = sum(pad[1 + dy:1 + dy + nc[1], 1 + dx:1 + dx + nc[0]] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    return int((cnt * win).sum())


def test_candidate_counts_of_both_grids(rbf):
    p = W.lattice_problem(120, 0.85, seed=72)
    cfg = rbf.config_for(p, mixed=True, factor_precision=rbf.RBF_FP32, inner_cutoff=6.1)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    assert rbf.rbf_count_candidates(ctx.handle, 0) == host_candidates(p.xy, p.cutoff)
    with pytest.raises(rbf.RbfError):
        rbf.rbf_count_candidates(ctx.handle, 1)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, _ = ctx.solve(dev(p.f), w, cfg)
    assert st == 0
    got = rbf.rbf_count_candidates(ctx.handle, 1)
    assert got == host_candidates(p.xy, min(6.1 * p.sigma, p.cutoff))
    assert got < rbf.rbf_count_candidates(ctx.handle, 0)
    ctx.close()


def inner_apply(rbf, p, w, variant, ri=6.1):
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_debug_inner_matvec(ctx.handle, ri, dev(w), y, variant)
    out = host(y)
    ctx.close()
    return out


@pytest.mark.parametrize("n_side,ratio", [(96, 0.8), (130, 0.6), (64, 1.0), (37, 0.9)])
def test_symmetric_inner_operator(rbf, n_side, ratio):
    """The symmetric FP32 kernel (each neighbouring cell pair once) against the
    stencil kernel (every target against its 3 x 3 cells), and both against the
    oracle's FP64 matvec truncated at the inner cutoff: the pairs of the stencil
    beyond r_i, which the FP32 operator keeps, are each below e^-18.6."""
    p = W.lattice_problem(n_side, ratio, seed=400 + n_side)
    w = np.random.default_rng(9).standard_normal(p.n)
    ys = inner_apply(rbf, p, w, 0)
    yt = inner_apply(rbf, p, w, 1)
    scale = np.max(np.abs(yt))
    assert np.max(np.abs(ys - yt)) <= 1e-5 * scale
    ri = 6.1 * p.sigma
    ref = O.matvec_cutoff(p.xy, w.astype(np.float32).astype(np.float64), p.sigma, ri, c=ri)
    assert np.max(np.abs(ys - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_symmetric_inner_operator_random_points_and_dense_cells(rbf):
    """Uneven cells (uniform random points, including empty cells); and a
    clump whose inner cell exceeds 128 points, which the symmetric kernel
    refuses (the solver then keeps the stencil kernel)."""
    rng = np.random.default_rng(10)
    xy = np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(6000, 2)))
    from dataclasses import replace
    base = W.lattice_problem(8, 0.8, seed=1)
    p = replace(base, xy=xy, f=np.zeros(6000), sigma=0.02, cutoff=0.172)
    w = rng.standard_normal(p.n)
    ys, yt = inner_apply(rbf, p, w, 0), inner_apply(rbf, p, w, 1)
    assert np.max(np.abs(ys - yt)) <= 1e-5 * np.max(np.abs(yt))
    clump = np.ascontiguousarray(np.vstack([rng.uniform(0.0, 0.05, size=(300, 2)), xy[:500]]))
    q = replace(p, xy=clump, f=np.zeros(clump.shape[0]))
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, dev(q.xy), q.n, rbf.RbfParams(q.sigma, q.cutoff, 0.0, 0))
    y = torch.empty(q.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_debug_inner_matvec(ctx.handle, 6.1, dev(rng.standard_normal(q.n)), y, 0)
    assert e.value.status == 8
    rbf.rbf_debug_inner_matvec(ctx.handle, 6.1, dev(rng.standard_normal(q.n)), y, 1)
    ctx.close()
