"""Batches of independent problems in one context: every problem of the batch
must give what the oracle gives for it alone (bit-exact index work, FP64 matvec
within 1e-13, solves to a true relative residual <= 1e-13), and a problem's
solution must not depend on the other problems of the batch."""
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


def small_batch():
    sizes = [(2, 0.9), (3, 1.0), (16, 0.8), (21, 0.95), (33, 0.85), (12, 0.8), (40, 0.9)]
    return [W.lattice_problem(n, r, seed=100 + k, rhs="four_gaussians") for k, (n, r) in enumerate(sizes)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup(rbf, probs, factor_precision=0, sym64=0):
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs, factor_precision=factor_precision)
    ctx = rbf.Context(0)
    rbf.rbf_set_option(ctx.handle, rbf.RBF_OPT_SYMMETRIC_F64, sym64)
    rbf.rbf_bin_batch(ctx.handle, dev(xy), ptr, params)
    rbf.rbf_rasm_setup_batch(ctx.handle, rasm)
    return ctx, xy, f, ptr


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batch_binning_and_lists_match_each_problem_alone(rbf):
    probs = small_batch()
    ctx, xy, f, ptr = setup(rbf, probs)
    n = ptr[-1]
    pd = torch.empty(n, dtype=torch.int32, device="cuda")
    rbf.rbf_get_bins(ctx.handle, pd, None)
    perm = host(pd)
    nsub_tot, _, ct, ot = rbf.rbf_get_subdomain_sizes(ctx.handle)
    cp = torch.empty(nsub_tot + 1, dtype=torch.int32, device="cuda")
    op = torch.empty(nsub_tot + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(ct, dtype=torch.int32, device="cuda")
    oi = torch.empty(ot, dtype=torch.int32, device="cuda")
    rbf.rbf_get_subdomains(ctx.handle, cp, ci, op, oi)
    cp, ci, op, oi = host(cp), host(ci), host(op), host(oi)
    sub0 = 0
    for b, p in enumerate(probs):
        lo, hi = ptr[b], ptr[b + 1]
        _, rperm, _ = O.bin_points(p.xy, p.cutoff)
        np.testing.assert_array_equal(perm[lo:hi] - lo, rperm)
        (nbx, nby), rcp, rci, rop, roi = O.subdomains(p.xy, p.x0, p.x0, p.core_size, p.overlap)
        ns = nbx * nby
        np.testing.assert_array_equal(cp[sub0:sub0 + ns + 1] - cp[sub0], rcp)
        np.testing.assert_array_equal(ci[cp[sub0]:cp[sub0 + ns]] - lo, rci)
        np.testing.assert_array_equal(op[sub0:sub0 + ns + 1] - op[sub0], rop)
        np.testing.assert_array_equal(oi[op[sub0]:op[sub0 + ns]] - lo, roi)
        sub0 += ns
    assert sub0 == nsub_tot
    ctx.close()


def test_batch_matvec_and_rasm_per_problem(rbf):
    probs = small_batch()
    ctx, xy, f, ptr = setup(rbf, probs)
    n = ptr[-1]
    v = np.random.default_rng(3).standard_normal(n)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(v), y)
    rbf.rbf_rasm_apply(ctx.handle, dev(v), z)
    y, z = host(y), host(z)
    for b, p in enumerate(probs):
        lo, hi = ptr[b], ptr[b + 1]
        ref = O.matvec_cutoff(p.xy, v[lo:hi], p.sigma, p.cutoff)
        assert rel(y[lo:hi], ref) <= 1e-13
        pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
        assert rel(z[lo:hi], pr.rasm_apply(v[lo:hi])) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("sym64", [1, 0])
def test_batch_matvec_kernel_choice_is_per_problem(rbf, sym64):
    """With the symmetric FP64 matvec enabled it serves problems with cells as
    wide as r_c holding at most 160 points; a crowded problem (h/sigma = 0.6,
    about 205 points a cell) and one with cells of r_c / 2 take the stencil
    kernel. In one batch each problem gets the same bits as alone, and the
    oracle's values; likewise with the stencil kernel throughout."""
    probs = [W.lattice_problem(24, 0.9, seed=71), W.lattice_problem(20, 0.6, seed=72),
             W.lattice_problem(28, 0.85, seed=73), W.lattice_problem(17, 1.0, seed=74)]
    cells = [0.0, 0.0, 0.5 * probs[2].cutoff, 0.0]
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs)
    for b, c in enumerate(cells):
        params[b].cell_size = c
    ctx = rbf.Context(0)
    rbf.rbf_set_option(ctx.handle, rbf.RBF_OPT_SYMMETRIC_F64, sym64)
    rbf.rbf_bin_batch(ctx.handle, dev(xy), ptr, params)
    v = np.random.default_rng(8).standard_normal(ptr[-1])
    y = torch.empty(ptr[-1], dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(v), y)
    y = host(y)
    ctx.close()
    for b, p in enumerate(probs):
        lo, hi = ptr[b], ptr[b + 1]
        c1 = rbf.Context(0)
        rbf.rbf_set_option(c1.handle, rbf.RBF_OPT_SYMMETRIC_F64, sym64)
        rbf.rbf_bin_batch(c1.handle, dev(p.xy), [0, p.n], [params[b]])
        y1 = torch.empty(p.n, dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(c1.handle, dev(v[lo:hi]), y1)
        c1.close()
        np.testing.assert_array_equal(host(y1), y[lo:hi])
        ref = O.matvec_cutoff(p.xy, v[lo:hi], p.sigma, p.cutoff)
        assert np.max(np.abs(y[lo:hi] - ref)) <= 1e-13 * np.max(np.abs(ref))


def solve_batch(rbf, probs, mixed=False, repeat=1, sym64=0):
    ctx, xy, f, ptr = setup(rbf, probs, factor_precision=1 if mixed else 0, sym64=sym64)
    sp = rbf.RbfSolveParams(1e-13, 30, 20000, int(mixed), 60, 1e-5)
    outs = []
    for _ in range(repeat):
        w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
        st, infos = rbf.rbf_solve_batch(ctx.handle, dev(f), w, sp, len(probs), check=False)
        outs.append(host(w))
    ctx.close()
    return st, infos, outs, ptr


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_solve_reaches_tolerance_per_problem(rbf, mixed):
    probs = small_batch()
    st, infos, (w,), ptr = solve_batch(rbf, probs, mixed)
    assert st == 0, [i.as_dict() for i in infos]
    for b, p in enumerate(probs):
        wb = w[ptr[b]:ptr[b + 1]]
        r = p.f - O.matvec_cutoff(p.xy, wb, p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13, (b, infos[b].as_dict())
        assert infos[b].relres <= 1e-13


def test_batch_result_independent_of_the_mix(rbf):
    """Each problem's w is bit-identical alone and inside the batch, and the
    batch result is reproducible run to run."""
    probs = small_batch()
    _, _, (w1, w2), ptr = solve_batch(rbf, probs, repeat=2)
    np.testing.assert_array_equal(w1, w2)
    for b in (1, 4, 6):
        _, _, (wa,), _ = solve_batch(rbf, [probs[b]])
        np.testing.assert_array_equal(wa, w1[ptr[b]:ptr[b + 1]])


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_with_symmetric_f64_matvec(rbf, mixed):
    """The symmetric FP64 matvec inside the solver (captured cycles, batch
    compaction): every problem converges and gets the same bits alone as in
    the batch."""
    probs = small_batch()[2:7]
    st, infos, (w,), ptr = solve_batch(rbf, probs, mixed, sym64=1)
    assert st == 0
    for b, p in enumerate(probs):
        assert infos[b].status == 0 and infos[b].relres <= 1e-13, infos[b].as_dict()
    for b in (0, 3, 4):
        _, _, (wa,), _ = solve_batch(rbf, [probs[b]], mixed, sym64=1)
        np.testing.assert_array_equal(wa, w[ptr[b]:ptr[b + 1]])


def test_single_solver_equals_batch_of_one(rbf):
    p = W.lattice_problem(30, 0.85, seed=7)
    _, _, (wb,), _ = solve_batch(rbf, [p])
    cfg = rbf.config_for(p)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg)
    np.testing.assert_array_equal(host(w), wb)
    ctx.close()


def test_batch_rejects_single_problem_calls(rbf):
    probs = small_batch()[:3]
    ctx, xy, f, ptr = setup(rbf, probs)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_solve(ctx.handle, dev(f), w, rbf.RbfSolveParams(1e-13, 30, 100, 0, 0, 0.0))
    assert e.value.status == 8
    ctx.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_stagnating_problem_stops_alone(rbf, mixed):
    """h/sigma = 0.6 with 4x4-point subdomains stalls near a relative residual
    of 0.44 (the oracle's GMRES on the same problem stays above 0.43 for 3000
    steps): it is stopped on its own with status NOT_CONVERGED and the flag
    set, while the other problems converge exactly as they do alone."""
    probs = small_batch()[2:5]
    hard = W.lattice_problem(24, 0.6, seed=5, rhs="four_gaussians")
    mix = probs[:1] + [hard] + probs[1:]
    st, infos, (w,), ptr = solve_batch(rbf, mix, mixed)
    assert st == 6
    hi = infos[1]
    assert hi.stagnated == 1 and hi.status == 6, hi.as_dict()
    assert 0.3 < hi.relres < 1.0 and hi.iters < 400
    for b in (0, 2, 3):
        assert infos[b].status == 0 and infos[b].stagnated == 0, infos[b].as_dict()
        _, _, (wa,), _ = solve_batch(rbf, [mix[b]], mixed)
        np.testing.assert_array_equal(wa, w[ptr[b]:ptr[b + 1]])


def test_single_solver_stops_on_stagnation(rbf):
    p = W.lattice_problem(24, 0.6, seed=5, rhs="four_gaussians")
    cfg = rbf.config_for(p)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 6 and info.status == 6 and info.stagnated == 1, info.as_dict()
    assert info.iters < 400
    ctx.close()


def test_batch_honours_max_iters_mid_cycle(rbf):
    """A step cap inside a cycle stops every problem exactly there, as the
    single-problem solver does (same iterate, bit for bit)."""
    p = W.lattice_problem(30, 0.85, seed=7)
    for cap in (17, 45):
        ctx, xy, f, ptr = setup(rbf, [p])
        wb = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        sp = rbf.RbfSolveParams(1e-13, 30, cap, 0, 0, 0.0)
        st, infos = rbf.rbf_solve_batch(ctx.handle, dev(f), wb, sp, 1, check=False)
        ctx.close()
        assert st == 6 and infos[0].iters == cap
        cfg = rbf.config_for(p, max_iters=cap)
        c1 = rbf.Context(0)
        c1.bin(dev(p.xy), cfg)
        c1.rasm_setup(cfg)
        w1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st1, info1 = c1.solve(dev(p.f), w1, cfg, check=False)
        c1.close()
        assert info1.iters == cap
        np.testing.assert_array_equal(host(w1), host(wb))


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_tail_after_compaction_matches_alone(rbf, mixed):
    """Seven quick problems and one slow one: once the quick ones stop, the
    batch restricts its work lists to the slow problem and captures its cycle
    again; every problem still gives the same bits alone and in the batch."""
    probs = [W.lattice_problem(8 + k, 1.0, seed=300 + k, rhs="four_gaussians") for k in range(7)]
    probs.append(W.lattice_problem(40, 0.75, seed=310, rhs="four_gaussians"))
    st, infos, (wb,), ptr = solve_batch(rbf, probs, mixed)
    assert st == 0, [i.as_dict() for i in infos]
    assert infos[-1].iters > max(i.iters for i in infos[:-1])   # the tail runs alone
    for b in (0, 3, 7):
        _, _, (wa,), _ = solve_batch(rbf, [probs[b]], mixed)
        np.testing.assert_array_equal(wa, wb[ptr[b]:ptr[b + 1]])


def config4_slice():
    """A seeded slice of the 4096-problem batch workload (the same (n_side, h/sigma)
    draws and per-problem seeds as the full batch): its largest problem at
    h/sigma >= 0.7 (128 x 128 = 16,384 points) and eleven others drawn at random,
    all at h/sigma >= 0.7 (below it the 4 x 4-point subdomains stall GMRES)."""
    sizes = W.batch_problem_sizes(4096, 256, 16384, W.DEFAULT_SEED)
    big = int(np.argmax([s[0] if s[1] >= 0.7 else 0 for s in sizes]))
    rng = np.random.default_rng(77)
    pick = [big]
    for k in rng.permutation(len(sizes)):
        if len(pick) == 12:
            break
        if int(k) != big and sizes[k][1] >= 0.7:
            pick.append(int(k))
    return [W.lattice_problem(sizes[k][0], sizes[k][1], seed=W.DEFAULT_SEED + 1 + k, rhs="four_gaussians")
            for k in pick]


def test_config4_slice_matches_oracle_per_problem(rbf):
    """Mixed batched solve (FP32 inner on the 6.1 sigma grid, FP64 outer) of the
    slice: every problem reaches a true relative residual <= 1e-13, recomputed
    by the oracle's FP64 matvec, and its w agrees with the oracle's own FP64
    solve of that problem alone to within the conditioning of the system."""
    probs = config4_slice()
    assert max(p.n for p in probs) == 128 * 128
    ctx, xy, f, ptr = setup(rbf, probs, factor_precision=1)
    sp = rbf.RbfSolveParams(1e-13, 30, 3000, 1, 3000, 1e-5, 6.1)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    st, infos = rbf.rbf_solve_batch(ctx.handle, dev(f), w, sp, len(probs), check=False)
    w = host(w)
    ctx.close()
    assert st == 0, [i.as_dict() for i in infos]
    for b, p in enumerate(probs):
        wb = w[ptr[b]:ptr[b + 1]]
        r = p.f - O.matvec_cutoff(p.xy, wb, p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13, (b, infos[b].as_dict())
        pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
        wo, oi = pr.solve(p.f, max_iters=3000)
        assert oi.relres <= 1e-13
        # two solutions of one SPD system, each to 1e-13: |dw| / |w| <= cond * 2e-13
        assert rel(wb, wo) <= 1e-5, (b, p.n, p.h / p.sigma)
