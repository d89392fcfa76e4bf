"""Injected failures, made on the host: non-finite inputs, a device-memory cap
that forces the out-of-memory paths, and the recovery of a context after
each. None of these faults the GPU; every failure comes back as a status.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_5413_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INVALID_ARG, OOM, STATE = 1, 2, 8


@pytest.fixture(scope="module")
def rbf():
    from paper_0909_5413_gb300 import rbf as R
    R.load()
    return R


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_relres(p, w):
    r = p.f - O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    return float(np.linalg.norm(r) / np.linalg.norm(p.f))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_bin_rejects_non_finite_coordinates(rbf, bad):
    p = W.lattice_problem(30, 0.8, seed=101)
    xy = p.xy.copy()
    xy[417, 1] = bad
    ctx = rbf.Context(0)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_bin(ctx.handle, dev(xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    assert e.value.status == INVALID_ARG
    assert "non-finite" in str(e.value)
    # the context is usable afterwards: the clean input bins and multiplies like the oracle
    rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    w = np.random.default_rng(1).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_matvec(ctx.handle, dev(w), y)
    torch.cuda.synchronize()
    ref = O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))
    ctx.close()


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_solve_rejects_non_finite_rhs(rbf, mixed, bad):
    p = W.lattice_problem(32, 0.8, seed=102)
    cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64)
    ctx = rbf.Context(0)
    ctx.bin(dev(p.xy), cfg)
    ctx.rasm_setup(cfg)
    f = p.f.copy()
    f[5] = bad
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, _ = ctx.solve(dev(f), w, cfg, check=False)
    assert st == INVALID_ARG
    # the same context then solves the clean problem to the oracle's residual
    w.zero_()
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 0
    torch.cuda.synchronize()
    assert oracle_relres(p, w.cpu().numpy()) <= 1e-13
    ctx.close()


def test_batch_solve_rejects_non_finite_rhs(rbf):
    probs = [W.lattice_problem(n, 0.8, seed=110 + n) for n in (20, 24, 28)]
    xy, f, ptr, params, rasm = rbf.batch_arrays(probs)
    f = f.copy()
    f[ptr[1] + 3] = np.nan
    ctx = rbf.Context(0)
    rbf.rbf_bin_batch(ctx.handle, dev(xy), ptr, params)
    rbf.rbf_rasm_setup_batch(ctx.handle, rasm)
    w = torch.zeros(ptr[-1], dtype=torch.float64, device="cuda")
    st, _ = rbf.rbf_solve_batch(ctx.handle, dev(f), w, rbf.RbfSolveParams(1e-13, 30, 3000, 0, 40, 1e-5, 0.0),
                                len(probs), check=False)
    assert st == INVALID_ARG
    ctx.close()


def test_memory_cap_forces_oom_in_setup_and_solve(rbf):
    """A cap below what the subdomain factors need makes rbf_rasm_setup return
    OOM; a cap that admits the setup but not the Krylov basis makes rbf_solve
    return OOM. Lifting the cap, the same context sets up and solves."""
    p = W.lattice_problem(96, 0.8, seed=103)
    cfg = rbf.config_for(p)
    ctx = rbf.Context(0)
    h = ctx.handle
    ctx.bin(dev(p.xy), cfg)
    held = rbf.rbf_device_bytes(h)
    rbf.rbf_set_memory_limit(h, held + 4096)
    with pytest.raises(rbf.RbfError) as e:
        ctx.rasm_setup(cfg)
    assert e.value.status == OOM
    assert "memory limit" in str(e.value)
    # enough for the factors, not for the 31 basis vectors of GMRES(30)
    rbf.rbf_set_memory_limit(h, 0)
    ctx.rasm_setup(cfg)
    held = rbf.rbf_device_bytes(h)
    rbf.rbf_set_memory_limit(h, held + 8 * p.n * 4)
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st, _ = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == OOM
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_set_memory_limit(h, -1)
    assert e.value.status == INVALID_ARG
    rbf.rbf_set_memory_limit(h, 0)
    w.zero_()
    st, info = ctx.solve(dev(p.f), w, cfg, check=False)
    assert st == 0
    torch.cuda.synchronize()
    assert oracle_relres(p, w.cpu().numpy()) <= 1e-13
    ctx.close()


def test_calls_out_of_order_report_state(rbf):
    p = W.lattice_problem(16, 0.8, seed=104)
    ctx = rbf.Context(0)
    v = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_matvec(ctx.handle, v, v)
    assert e.value.status == STATE
    cfg = rbf.config_for(p)
    ctx.bin(dev(p.xy), cfg)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_rasm_apply(ctx.handle, v, v)
    assert e.value.status == STATE
    st, _ = ctx.solve(dev(p.f), v, cfg, check=False)
    assert st == STATE
    ctx.close()
