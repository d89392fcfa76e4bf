"""The fused Arnoldi step of the batched mixed solver: one persistent
cooperative launch per step (apply, symmetric matvec, Gram-Schmidt, Arnoldi
column, scaling) with bounded grid-wide barriers. Its results must be the
separate kernels' bit for bit, and an expired barrier wait must come back as
RBF_ERR_TIMEOUT with the context still usable. The timeout is forced on the
host side of the contract: an option makes every barrier wait for one block
more than the grid has, with a short poll limit; nothing faults or hangs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_5413_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TIMEOUT = 7


@pytest.fixture(scope="module")
def rbf():
    from paper_0909_5413_gb300 import rbf as R
    R.load()
    return R


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problems():
    sizes = [(40, 0.9), (72, 0.8), (24, 1.0), (100, 0.85), (17, 0.95), (64, 0.75)]
    return [W.lattice_problem(n, r, seed=500 + k, rhs="four_gaussians") for k, (n, r) in enumerate(sizes)]


def solve(rbf, probs, fused, options=()):
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP32)
    ctx = rbf.Context(0)
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, int(fused))
    for opt, val in options:
        rbf.rbf_set_option(h, opt, val)
    rbf.rbf_bin_batch(h, dev(xy), ptr, params)
    rbf.rbf_rasm_setup_batch(h, rasm)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    sp = rbf.RbfSolveParams(1e-13, 30, 3000, 1, 200, 1e-5, 6.1)
    l0 = ctx.launches
    st, infos = rbf.rbf_solve_batch(h, dev(f), w, sp, len(probs), check=False)
    torch.cuda.synchronize()
    launches = ctx.launches - l0
    return ctx, st, infos, w.cpu().numpy(), ptr, launches


def test_fused_step_matches_separate_kernels_bit_for_bit(rbf):
    probs = problems()
    c1, st1, inf1, w1, ptr, l1 = solve(rbf, probs, 1)
    c0, st0, inf0, w0, _, l0 = solve(rbf, probs, 0)
    c2, st2, inf2, w2, _, _ = solve(rbf, probs, 2)   # adaptive: six problems, all in the fused tail
    c1.close()
    c0.close()
    c2.close()
    assert st1 == 0 and st0 == 0 and st2 == 0, [i.as_dict() for i in inf1]
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(w2, w0)
    assert [i.iters for i in inf1] == [i.iters for i in inf0]
    assert l1 * 3 < l0, (l1, l0)   # one launch per step instead of about ten
    for b, p in enumerate(probs):
        wb = w1[ptr[b]:ptr[b + 1]]
        r = p.f - O.matvec_cutoff(p.xy, wb, p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13


def test_fused_step_barrier_timeout_is_reported_and_recoverable(rbf):
    probs = problems()[:3]
    ctx, st, infos, _, _, _ = solve(rbf, probs, 1, options=((rbf.RBF_OPT_BARRIER_SPIN_LIMIT, 2000),
                                                              (rbf.RBF_OPT_BARRIER_EXTRA_BLOCK, 1)))
    assert st == TIMEOUT
    assert "gave up waiting" in rbf.load().rbf_last_error(ctx.handle).decode()
    # the same context, back to the default barrier: the batch solves to the oracle's tolerance
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_BARRIER_EXTRA_BLOCK, 0)
    rbf.rbf_set_option(h, rbf.RBF_OPT_BARRIER_SPIN_LIMIT, 1 << 23)
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP32)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    sp = rbf.RbfSolveParams(1e-13, 30, 3000, 1, 200, 1e-5, 6.1)
    st, infos = rbf.rbf_solve_batch(h, dev(f), w, sp, len(probs), check=False)
    assert st == 0, [i.as_dict() for i in infos]
    wh = w.cpu().numpy()
    for b, p in enumerate(probs):
        r = p.f - O.matvec_cutoff(p.xy, wh[ptr[b]:ptr[b + 1]], p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13
    ctx.close()


def test_options_are_validated(rbf):
    ctx = rbf.Context(0)
    for opt, val in ((99, 0), (rbf.RBF_OPT_FUSED_STEP, 3), (rbf.RBF_OPT_BARRIER_SPIN_LIMIT, 0)):
        with pytest.raises(rbf.RbfError) as e:
            rbf.rbf_set_option(ctx.handle, opt, val)
        assert e.value.status == 1
    ctx.close()


def test_fused_step_matches_separate_kernels_with_segmented_reductions(rbf):
    """A problem of more than 2047 chunks (8.4 M points) has its chunk partials
    summed in several segments, by one warp each in the separate kernels and in
    sequence in the fused step: the same bits either way, next to small
    problems of one segment."""
    probs = [W.lattice_problem(2900, 0.9, seed=560, rhs="four_gaussians"),
             W.lattice_problem(40, 0.85, seed=561, rhs="four_gaussians"),
             W.lattice_problem(23, 1.0, seed=562, rhs="four_gaussians")]
    assert probs[0].n > 2048 * 4096
    c1, st1, inf1, w1, ptr, _ = solve(rbf, probs, 1)
    c0, st0, inf0, w0, _, _ = solve(rbf, probs, 0)
    c1.close()
    c0.close()
    assert st1 == 0 and st0 == 0, [i.as_dict() for i in inf0]
    np.testing.assert_array_equal(w1, w0)
    assert all(i.relres <= 1e-13 for i in inf0)
    for b in (1, 2):
        wb = w0[ptr[b]:ptr[b + 1]]
        r = probs[b].f - O.matvec_cutoff(probs[b].xy, wb, probs[b].sigma, probs[b].cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(probs[b].f) <= 1e-13


@pytest.mark.parametrize("n_side,fused_by_default", [(90, True), (600, False)])
def test_single_problem_default_takes_fused_step_when_small(rbf, n_side, fused_by_default):
    """The default (adaptive) mode runs a single problem of at most 262,144
    points on the fused step and a larger one on the separate kernels; either
    way the bits are those of the separate kernels."""
    p = W.lattice_problem(n_side, 0.85, seed=570 + n_side, rhs="four_gaussians")
    c2, st2, i2, w2, ptr, l2 = solve(rbf, [p], 2)
    c0, st0, i0, w0, _, l0 = solve(rbf, [p], 0)
    c2.close()
    c0.close()
    assert st2 == 0 and st0 == 0
    np.testing.assert_array_equal(w2, w0)
    if fused_by_default:
        assert l2 * 3 < l0, (l2, l0)
    else:
        assert l2 == l0
