"""rbf_matvec_noalloc: the FP64 matvec for callers that cannot let a library
allocate device memory (real-time loops that must avoid the allocator's
implicit synchronisation, applications whose device memory belongs to another
framework's pool). Called through the C ABI, it must give what rbf_matvec
gives and what the CPU oracle gives, on two calls in a row (the shared static
scratch keeps the previous call's data), hold no device memory of its own,
and refuse point sets larger than its fixed scratch.

This file is collected last on purpose; it needs nothing from the others and
passes alone in a fresh process too."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0909_5413_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_matvec_matches_matvec_twice():
    from paper_0909_5413_gb300 import rbf
    p = W.lattice_problem(300, 0.8, seed=31)        # 90,000 points, many blocks and a ragged tail
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, torch.from_numpy(p.xy).cuda(), p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    rng = np.random.default_rng(5)
    for call in range(2):
        w_h = rng.standard_normal(p.n)
        w = torch.from_numpy(w_h).cuda()
        y_ref = torch.empty(p.n, dtype=torch.float64, device="cuda")
        y_na = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(ctx.handle, w, y_ref, rbf.RBF_FP64)
        rbf.rbf_matvec_noalloc(ctx.handle, w, y_na)
        torch.cuda.synchronize()
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert rel_err(a, b) <= 1e-13, call
        ref = O.matvec_cutoff(p.xy, w_h, p.sigma, p.cutoff)
        assert rel_err(a, ref) <= 1e-13, call
        assert max_rel(a, ref) <= 1e-13, call
    ctx.close()


def test_noalloc_on_a_fresh_context_holds_no_memory():
    """A context that has only been binned: the no-alloc matvec alone, two calls
    in a row, against the oracle and against rbf_matvec on a second context;
    neither the context's device bytes nor the device's free memory move."""
    from paper_0909_5413_gb300 import rbf
    p = W.lattice_problem(257, 0.8, seed=33)        # 66,049 points
    xy = torch.from_numpy(p.xy).cuda()
    ctx = rbf.Context(0)
    rbf.rbf_bin(ctx.handle, xy, p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    rng = np.random.default_rng(9)
    w_hs = [rng.standard_normal(p.n) for _ in range(3)]
    ws = [torch.from_numpy(a).cuda() for a in w_hs]
    ys = [torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    rbf.rbf_matvec_noalloc(ctx.handle, ws[0], ys[0])   # first call in this process may load the kernels
    torch.cuda.synchronize()
    bytes0 = rbf.rbf_device_bytes(ctx.handle)
    free0, _ = torch.cuda.mem_get_info()
    for k in (1, 2):
        rbf.rbf_matvec_noalloc(ctx.handle, ws[k], ys[k])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rbf.rbf_device_bytes(ctx.handle) == bytes0
    assert free1 == free0
    other = rbf.Context(0)
    rbf.rbf_bin(other.handle, xy, p.n, rbf.RbfParams(p.sigma, p.cutoff, 0.0, 0))
    for k in range(3):
        got = ys[k].cpu().numpy()
        ref = O.matvec_cutoff(p.xy, w_hs[k], p.sigma, p.cutoff)
        assert rel_err(got, ref) <= 1e-13, k
        assert max_rel(got, ref) <= 1e-13, k
        y2 = torch.empty(p.n, dtype=torch.float64, device="cuda")
        rbf.rbf_matvec(other.handle, ws[k], y2, rbf.RBF_FP64)
        torch.cuda.synchronize()
        assert rel_err(got, y2.cpu().numpy()) <= 1e-13, k
    other.close()
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
