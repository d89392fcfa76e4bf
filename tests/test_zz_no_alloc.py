"""rbf_matvec_noalloc: the FP64 matvec for callers that cannot allocate device
memory (graph capture, real-time loops, memory owned by another framework's
pool). Called through the C ABI, it must give what rbf_matvec gives, on two
calls in a row (the shared static scratch keeps the previous call's data), and
refuse point sets larger than its fixed scratch.

This file is collected last on purpose; it needs nothing from the others and
passes alone in a fresh process too."""
import numpy as np
import pytest

from paper_0909_5413_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matvec_matches_matvec_twice():
    from paper_0909_5413_gb300 import rbf
    p = W.lattice_problem(300, 0.8, seed=31)        # 90,000 points, many blocks and a ragged tail
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, torch.from_numpy(p.xy).cuda(), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    rng = np.random.default_rng(5)
    for call in range(2):
        w = torch.from_numpy(rng.standard_normal(p.n)).cuda()
        y_ref = torch.empty(p.n, dtype=torch.float64, device="cuda")
        y_na = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(ctx.handle, w, y_ref, rbf.RBF_FP64)
        rbf.rbf_matvec_noalloc(ctx.handle, w, y_na)
        torch.cuda.synchronize()
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert rel_err(a, b) <= 1e-13, call
    ctx.close()


def test_noalloc_rejects_oversize_point_sets():
    from paper_0909_5413_gb300 import rbf
    xy, h = W.jittered_lattice(1025, seed=32)        # 1,050,625 points > 2^20
    xy = xy[: (1 << 20) + 1].copy()
    ctx = rbf.Context(0)
    sigma = h / 0.8
    rbf.rbf_bin(ctx.handle, torch.from_numpy(xy).cuda(), xy.shape[0], rbf.RbfParams(sigma, 8.6 * sigma, 0.0, 0))
    w = torch.zeros(xy.shape[0], dtype=torch.float64, device="cuda")
    y = torch.zeros_like(w)
    with pytest.raises(rbf.RbfError) as e:
        rbf.rbf_matvec_noalloc(ctx.handle, w, y)
    assert e.value.status == 1
    assert "static scratch capacity" in str(e.value)
    ctx.close()
