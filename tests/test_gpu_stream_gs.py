"""The FP32 Gram-Schmidt passes of the mixed form with the basis streamed
through shared memory by bulk asynchronous copies: the same bits as the
register passes (single problems and batches, separate kernels and the fused
step), the oracle's residual at the end, and an expired copy wait reported as
RBF_ERR_TIMEOUT with the context still usable. The timeout is forced on the
host side of the contract: an option makes every wait poll a barrier that no
copy completes, with nothing copied; nothing faults or hangs."""
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


def solve(rbf, probs, options=()):
    """Mixed solve of a batch on the separate kernels (the passes under test)
    unless the options choose the fused step."""
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP32)
    ctx = rbf.Context(0)
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, 0)
    for opt, val in options:
        rbf.rbf_set_option(h, opt, val)
    rbf.rbf_bin_batch(h, dev(xy), ptr, params)
    rbf.rbf_rasm_setup_batch(h, rasm)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    sp = rbf.RbfSolveParams(1e-13, 30, 3000, 1, 200, 1e-5, 6.1)
    st, infos = rbf.rbf_solve_batch(h, dev(f), w, sp, len(probs), check=False)
    torch.cuda.synchronize()
    return ctx, st, infos, w.cpu().numpy(), ptr


def residual_ok(probs, w, ptr):
    for b, p in enumerate(probs):
        r = p.f - O.matvec_cutoff(p.xy, w[ptr[b]:ptr[b + 1]], p.sigma, p.cutoff)
        assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13


@pytest.mark.parametrize("n_side,ratio", [(130, 0.8), (67, 0.9), (300, 0.85)])
def test_streamed_passes_single_problem_bit_for_bit(rbf, n_side, ratio):
    """A single problem (chunks of 4096 elements from index 0, a ragged last
    chunk): streamed and register passes give the same w."""
    p = W.lattice_problem(n_side, ratio, seed=800 + n_side, rhs="four_gaussians")
    c1, st1, i1, w1, ptr = solve(rbf, [p])
    c0, st0, i0, w0, _ = solve(rbf, [p], options=((rbf.RBF_OPT_STREAM_GS, 0),))
    c1.close()
    c0.close()
    assert st1 == 0 and st0 == 0, (i1[0].as_dict(), i0[0].as_dict())
    np.testing.assert_array_equal(w1, w0)
    assert i1[0].iters == i0[0].iters
    residual_ok([p], w1, ptr)


def test_streamed_passes_batch_bit_for_bit(rbf):
    """A batch on the separate kernels: problems start at offsets that are not
    multiples of four elements, so the copies are widened to 16-byte
    boundaries and read from an offset; same bits as the register passes and
    as the fused step."""
    sizes = [(41, 0.9), (73, 0.8), (23, 1.0), (101, 0.85), (17, 0.95), (63, 0.75)]
    probs = [W.lattice_problem(n, r, seed=820 + k, rhs="four_gaussians") for k, (n, r) in enumerate(sizes)]
    assert any(p.n % 4 for p in probs)
    sep = (rbf.RBF_OPT_FUSED_STEP, 0)
    c1, st1, i1, w1, ptr = solve(rbf, probs, options=(sep,))
    c0, st0, i0, w0, _ = solve(rbf, probs, options=(sep, (rbf.RBF_OPT_STREAM_GS, 0)))
    c2, st2, i2, w2, _ = solve(rbf, probs, options=((rbf.RBF_OPT_FUSED_STEP, 1),))
    for c in (c0, c1, c2):
        c.close()
    assert st1 == 0 and st0 == 0 and st2 == 0
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(w1, w2)
    residual_ok(probs, w1, ptr)


def test_streamed_copy_timeout_is_reported_and_recoverable(rbf):
    p = W.lattice_problem(90, 0.85, seed=840, rhs="four_gaussians")
    ctx, st, infos, _, ptr = solve(rbf, [p], options=((rbf.RBF_OPT_BARRIER_SPIN_LIMIT, 2000),
                                                      (rbf.RBF_OPT_STREAM_WAIT_CHECK, 1)))
    assert st == TIMEOUT
    assert "did not arrive" in rbf.load().rbf_last_error(ctx.handle).decode()
    # the same context with the waits back to normal solves to the oracle's tolerance
    h = ctx.handle
    rbf.rbf_set_option(h, rbf.RBF_OPT_STREAM_WAIT_CHECK, 0)
    rbf.rbf_set_option(h, rbf.RBF_OPT_BARRIER_SPIN_LIMIT, 1 << 23)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    sp = rbf.RbfSolveParams(1e-13, 30, 3000, 1, 200, 1e-5, 6.1)
    st, infos = rbf.rbf_solve_batch(h, dev(p.f), w, sp, 1, check=False)
    assert st == 0, infos[0].as_dict()
    residual_ok([p], w.cpu().numpy(), ptr)
    ctx.close()


def test_stream_options_are_validated(rbf):
    ctx = rbf.Context(0)
    for opt in (rbf.RBF_OPT_STREAM_GS, rbf.RBF_OPT_STREAM_WAIT_CHECK):
        with pytest.raises(rbf.RbfError) as e:
            rbf.rbf_set_option(ctx.handle, opt, 2)
        assert e.value.status == 1
    ctx.close()
