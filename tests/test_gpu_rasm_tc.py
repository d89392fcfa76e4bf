"""FP32 subdomain inverses on the tensor cores (rbf_rasm_params.precision =
RBF_FP32): the block sweep with 3xTF32 MMAs, checked against the CPU oracle's
RASM (Eq. rasm) and additive Schwarz (Eq. asm) applies, the FP64 fallback for
subdomains it does not take, and the cost in inner steps of the mixed solve
against inverses computed in FP64."""
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


def apply_gpu(rbf, p, precision, additive=False, max_sub=0, ring_points=1):
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, dev(p.xy), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    rbf.rbf_rasm_setup(ctx.handle, rbf.RbfRasmParams(p.x0, p.x0, p.core_size, p.overlap, max_sub, precision,
                                                     int(additive)))
    counts = rbf.rbf_rasm_factor_counts(ctx.handle)
    v = np.random.default_rng(21).standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    rbf.rbf_rasm_apply(ctx.handle, dev(v), z)
    torch.cuda.synchronize()
    out = z.cpu().numpy()
    ctx.close()
    return v, out, counts


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("ratio,tol", [(1.0, 2e-4), (0.9, 1e-3), (0.8, 3e-3)])
def test_tensor_core_rasm_matches_oracle(rbf, ratio, tol):
    p = W.lattice_problem(45, ratio, seed=201)       # 2,025 points, ragged last row of boxes
    v, z, (tc, f64) = apply_gpu(rbf, p, rbf.RBF_FP32)
    assert f64 == 0 and tc > 100                     # every 6 x 6-point subdomain on the tensor cores
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    ref = pr.rasm_apply(v)
    assert max_rel(z, ref) <= tol


def test_tensor_core_additive_schwarz_matches_oracle(rbf):
    """Eq. asm keeps every row of A_i^{-1}: the sweep's full inverse."""
    p = W.lattice_problem(40, 0.9, seed=202)
    v, z, (tc, f64) = apply_gpu(rbf, p, rbf.RBF_FP32, additive=True)
    assert f64 == 0 and tc > 0
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap, additive=True)
    assert max_rel(z, pr.rasm_apply(v)) <= 1e-3


def test_large_subdomains_fall_back_to_fp64(rbf):
    """A ring of two lattice points makes 8 x 8 = 64-point overlap lists (over
    the 48 of the tensor-core path) inside the lattice: those are inverted in
    FP64, the smaller edge and corner subdomains on the tensor cores."""
    p = W.lattice_problem(40, 0.9, seed=203, ring_points=2)
    v, z, (tc, f64) = apply_gpu(rbf, p, rbf.RBF_FP32)
    assert f64 > 0 and tc > 0
    pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
    assert max_rel(z, pr.rasm_apply(v)) <= 1e-3
    # FP64 and FP64-then-rounded setups report every subdomain as FP64
    _, _, (tc2, f2) = apply_gpu(rbf, p, rbf.RBF_FP32_FROM_FP64)
    assert tc2 == 0 and f2 == tc + f64


@pytest.mark.parametrize("ratio", [0.8, 1.0])
def test_mixed_solve_with_tensor_core_inverses(rbf, ratio):
    """The mixed solve reaches the FP64 tolerance with tensor-core inverses
    (true residual by the oracle's matvec), in at most a few percent more inner
    steps than with inverses computed in FP64."""
    p = W.lattice_problem(160, ratio, seed=204)
    res = {}
    for prec in (rbf.RBF_FP32, rbf.RBF_FP32_FROM_FP64):
        cfg = rbf.config_for(p, mixed=True, factor_precision=prec, inner_cutoff=6.1)
        ctx = rbf.Context(0)
        ctx.bin(dev(p.xy), cfg)
        ctx.rasm_setup(cfg)
        w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = ctx.solve(dev(p.f), w, cfg, check=False)
        torch.cuda.synchronize()
        res[prec] = (st, info, w.cpu().numpy())
        ctx.close()
    st, info, w = res[rbf.RBF_FP32]
    assert st == 0, info.as_dict()
    r = p.f - O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    assert np.linalg.norm(r) / np.linalg.norm(p.f) <= 1e-13
    ref_iters = res[rbf.RBF_FP32_FROM_FP64][1].iters
    assert res[rbf.RBF_FP32_FROM_FP64][0] == 0
    assert info.iters <= 1.05 * ref_iters + 3, (info.iters, ref_iters)
