"""The FP64 matvec's pair values kept in device memory (RBF_OPT_STORE_F64):
computed once at the start of a solve, then replayed by every FP64 product
of that binning. The replay must give the stencil kernel's sums bit for bit
(solves and rbf_matvec), fall back to the matrix-free kernel when the values
do not fit under the context's memory limit, and follow a new binning."""
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


def run(rbf, p, store, mixed, limit=0, tile=0):
    """Solve p (store on or off) and one rbf_matvec after it. With `limit`,
    a first solve with the store off allocates the solver's workspace, then
    the context's memory limit leaves `limit` bytes of room and the store is
    switched on for the second solve."""
    cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64,
                         inner_cutoff=6.1 if mixed else 0.0)
    if tile:
        cfg.tile_f64 = tile
    ctx = rbf.Context(0)
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, 0 if limit else store)
    rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, 0)
    ctx.bin(dev(p.xy), cfg)
    pairs = rbf.rbf_count_pairs(h, 0)
    ctx.rasm_setup(cfg)
    fd = dev(p.f)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    if limit:
        st, info = ctx.solve(fd, w, cfg, check=False)
        assert st == 0
        rbf.rbf_set_memory_limit(h, rbf.rbf_device_bytes(h) + limit)
        rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, store)
        w.zero_()
    st, info = ctx.solve(fd, w, cfg, check=False)
    held = rbf.rbf_device_bytes(h)
    d = info.as_dict()
    d["store_bytes"] = rbf.rbf_store_f64_bytes(h)
    # a product after the solve (a replay when the values were kept)
    v = np.random.default_rng(4).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(h, dev(v), y)
    out = (st, d, host(w), host(y), v, held, pairs)
    ctx.close()
    return out


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("n_side,ratio", [(120, 0.8), (77, 0.95)])
def test_replay_matches_matrix_free_bit_for_bit(rbf, n_side, ratio, mixed):
    p = W.lattice_problem(n_side, ratio, seed=900 + n_side, rhs="four_gaussians")
    s1, i1, w1, y1, v, held1, pairs = run(rbf, p, 1, mixed)
    s0, i0, w0, y0, _, held0, _ = run(rbf, p, 0, mixed)
    assert s1 == 0 and s0 == 0, (i1, i0)
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(y1, y0)
    assert i1["iters"] == i0["iters"]
    # at least one FP64 value per nonzero of the truncated matrix is kept
    assert held1 - held0 >= i1["store_bytes"] >= 8 * pairs
    assert i0["store_bytes"] == 0
    ref = O.matvec_cutoff(p.xy, v, p.sigma, p.cutoff)
    assert np.max(np.abs(y1 - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_values_that_do_not_fit_stay_matrix_free(rbf):
    """A memory limit leaving 256 KB of room (the values need megabytes):
    nothing is kept, the same bits."""
    p = W.lattice_problem(100, 0.85, seed=950, rhs="four_gaussians")
    s1, i1, w1, y1, _, held1, pairs = run(rbf, p, 1, True, limit=1 << 18)
    s0, i0, w0, y0, _, held0, _ = run(rbf, p, 0, True)
    assert 8 * pairs > 1 << 20
    assert s1 == 0 and s0 == 0
    assert held1 - held0 < 1 << 18
    assert i1["store_bytes"] == 0
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(y1, y0)


@pytest.mark.parametrize("tile", [32, 64])
def test_replay_with_other_tiles(rbf, tile):
    p = W.lattice_problem(90, 0.8, seed=960, rhs="four_gaussians")
    s1, i1, w1, y1, _, held1, pairs = run(rbf, p, 1, False, tile=tile)
    s0, i0, w0, y0, _, held0, _ = run(rbf, p, 0, False, tile=tile)
    assert held1 - held0 >= 8 * pairs
    assert s1 == 0 and s0 == 0
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(y1, y0)


def test_kept_values_follow_a_new_binning(rbf):
    """Two problems binned one after the other in one context: each solve
    and product uses its own binning's values (the oracle's products)."""
    ctx = rbf.Context(0)
    for k, (n_side, ratio) in enumerate(((80, 0.9), (64, 0.8))):
        p = W.lattice_problem(n_side, ratio, seed=970 + k, rhs="four_gaussians")
        cfg = rbf.config_for(p)
        ctx.bin(dev(p.xy), cfg)
        assert rbf.rbf_store_f64_bytes(ctx.handle) == 0   # the previous binning's values are gone
        ctx.rasm_setup(cfg)
        w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = ctx.solve(dev(p.f), w, cfg, check=False)
        assert st == 0
        assert rbf.rbf_store_f64_bytes(ctx.handle) >= 8 * rbf.rbf_count_pairs(ctx.handle, 0)
        v = np.random.default_rng(k).standard_normal(p.n)
        y = torch.empty(p.n, dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(ctx.handle, dev(v), y)
        ref = O.matvec_cutoff(p.xy, v, p.sigma, p.cutoff)
        assert np.max(np.abs(host(y) - ref)) <= 1e-13 * np.max(np.abs(ref))
        r = p.f - O.matvec_cutoff(p.xy, host(w), p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13
    ctx.close()


def test_store_option_is_validated(rbf):
    ctx = rbf.Context(0)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_set_option(ctx.handle, rbf.RBF_OPT_STORE_F64, 2)
    assert e.value.status == 1
    ctx.close()


def test_switching_the_store_off_frees_it(rbf):
    p = W.lattice_problem(90, 0.85, seed=980, rhs="four_gaussians")
    cfg = rbf.config_for(p)
    ctx = rbf.Context(0)
    h = ctx.handle
    ctx.bin(dev(p.xy), cfg)
    pairs = rbf.rbf_count_pairs(h, 0)
    ctx.rasm_setup(cfg)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, _ = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 0
    held = rbf.rbf_device_bytes(h)
    assert rbf.rbf_store_f64_bytes(h) >= 8 * pairs
    rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, 0)
    assert held - rbf.rbf_device_bytes(h) >= 8 * pairs
    assert rbf.rbf_store_f64_bytes(h) == 0
    # matrix-free from here, the same bits
    v = dev(np.random.default_rng(5).standard_normal(p.n))
    y0 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(h, v, y0)
    rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, 1)
    w1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, _ = ctx.solve(dev(p.f), w1, cfg, check=False)
    assert st == 0
    y1 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(h, v, y1)
    np.testing.assert_array_equal(host(y0), host(y1))
    np.testing.assert_array_equal(host(w), host(w1))
    ctx.close()


@pytest.mark.parametrize("mixed", [True, False])
def test_where_the_values_are_kept(rbf, mixed):
    """A mixed solve keeps the values with its first outer residual product
    (formed in the same pass: one record of the profiler's store class, the
    other outer products replays); an FP64 solve keeps them at its start."""
    p = W.lattice_problem(100, 0.8, seed=990, rhs="four_gaussians")
    cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64,
                         inner_cutoff=6.1 if mixed else 0.0)
    ctx = rbf.Context(0)
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, 0)
    rbf.rbf_profile_enable(h, True)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    for k in range(rbf.RBF_PROF_COUNT):
        rbf.rbf_profile_read(h, k)   # only the solve's records below
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 0
    n_keep, t_keep = rbf.rbf_profile_read(h, rbf.RBF_PROF_STORE_F64)
    n_mv, _ = rbf.rbf_profile_read(h, rbf.RBF_PROF_MATVEC_F64)
    assert n_keep == 1 and t_keep > 0.0
    assert rbf.rbf_store_f64_bytes(h) >= 8 * rbf.rbf_count_pairs(h, 0)
    if mixed:
        outer = info.matvecs - info.iters   # w0 = 0: r0 = f needs no product
        assert outer == info.refinements >= 2
        assert n_mv == outer - 1
    # a second solve on the same binning keeps nothing more: every outer
    # product of a mixed solve is a replay
    w.zero_()
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 0
    n_keep, _ = rbf.rbf_profile_read(h, rbf.RBF_PROF_STORE_F64)
    n_mv, _ = rbf.rbf_profile_read(h, rbf.RBF_PROF_MATVEC_F64)
    assert n_keep == 0
    if mixed:
        assert n_mv == info.matvecs - info.iters
    rbf.rbf_profile_enable(h, False)
    ctx.close()
