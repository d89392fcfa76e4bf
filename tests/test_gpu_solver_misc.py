"""Solver details: the zero initial guess (r0 = f without a product), and the
profiler's class mask."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("mixed", [False, True])
def test_zero_initial_guess_skips_the_first_product(rbf, mixed):
    p = W.lattice_problem(48, 0.85, seed=91)
    cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg)
    assert st == 0 and info.relres <= 1e-13
    # one true residual per restart (refinement) and one at the end, less the first (r0 = f)
    outer = info.refinements if mixed else info.restarts
    assert info.matvecs == info.iters + outer
    # from the converged w (nonzero) the first residual is a product, and nothing else is needed
    st2, info2 = ctx.solve(dev(p.f), w, cfg)
    assert st2 == 0 and info2.iters == 0 and info2.matvecs == 1
    ctx.close()


def test_profiler_records_only_the_selected_classes(rbf):
    p = W.lattice_problem(40, 0.9, seed=92)
    cfg = rbf.config_for(p)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    h = ctx.handle
    rbf.rbf_profile_classes(h, 1 << rbf.RBF_PROF_MATVEC_F64)
    rbf.rbf_profile_enable(h, True)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, info = ctx.solve(dev(p.f), w, cfg)
    assert st == 0
    n_mv, t_mv = rbf.rbf_profile_read(h, rbf.RBF_PROF_MATVEC_F64)
    n_ap, _ = rbf.rbf_profile_read(h, rbf.RBF_PROF_RASM_APPLY)
    assert n_mv == info.matvecs and t_mv > 0.0 and n_ap == 0
    rbf.rbf_profile_classes(h, 0xFFFFFFFF)
    w.zero_()
    ctx.solve(dev(p.f), w, cfg)
    n_ap, t_ap = rbf.rbf_profile_read(h, rbf.RBF_PROF_RASM_APPLY)
    assert n_ap == info.applies and t_ap > 0.0
    rbf.rbf_profile_enable(h, False)
    ctx.close()
