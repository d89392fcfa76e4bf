"""Serving loop: requests of different sizes submitted together run
concurrently on their own slots, each result is bit-identical to the same
request solved alone and meets the tolerance against the CPU oracle, and
admission respects the device-memory budget."""
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


def requests(rbf, sizes, seed=300):
    out = []
    for k, (n_side, ratio, mixed) in enumerate(sizes):
        p = W.lattice_problem(n_side, ratio, seed=seed + k, rhs="four_gaussians")
        cfg = rbf.config_for(p, mixed=mixed, factor_precision=rbf.RBF_FP32 if mixed else rbf.RBF_FP64)
        out.append((p, cfg))
    return out


def oracle_relres(p, w):
    """True relative residual of w by the oracle's FP64 truncated matvec."""
    r = p.f - O.matvec_cutoff(p.xy, w, p.sigma, p.cutoff)
    return float(np.linalg.norm(r) / np.linalg.norm(p.f))


def alone(rbf, p, cfg):
    ctx = rbf.Context(0)
    w = np.zeros(p.n)
    st, info = ctx.interpolate_host(p.xy, p.f, w, cfg, check=False)
    ctx.close()
    return st, w


MIX = [(40, 0.9, True), (128, 0.85, False), (24, 1.0, False), (96, 0.8, True), (200, 0.95, True),
       (33, 0.75, False), (150, 0.9, False), (64, 0.8, True), (18, 0.9, True), (110, 1.0, True)]


def test_serve_results_identical_alone_and_in_the_mix(rbf):
    reqs = requests(rbf, MIX)
    srv = rbf.Server(0, slots=4)
    tickets = [srv.submit(p.xy, p.f, cfg) for p, cfg in reqs]
    results = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    spans = []
    for (p, cfg), (wst, r, w) in zip(reqs, results):
        assert wst == 0
        assert r.status == 0, r.info.as_dict()
        assert r.info.relres <= 1e-13
        st, wa = alone(rbf, p, cfg)
        assert st == 0
        np.testing.assert_array_equal(w, wa)
        # against the oracle: its own FP64 matvec gives the residual, and its own
        # solve of the request agrees to within the conditioning of the system
        assert oracle_relres(p, w) <= 1e-13
        if p.n <= 128 * 128:
            pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
            wo, oi = pr.solve(p.f, max_iters=3000)
            assert oi.relres <= 1e-13
            assert np.linalg.norm(w - wo) / np.linalg.norm(wo) <= 1e-5
        assert r.t_submit <= r.t_admit <= r.t_done
        spans.append((r.t_admit, r.t_done))
    # requests submitted together overlap on the device
    overlaps = sum(1 for i in range(len(spans)) for j in range(i) if spans[i][0] < spans[j][1] and
                   spans[j][0] < spans[i][1])
    assert overlaps > 0
    assert stats["completed"] == len(reqs) and stats["queued"] == 0 and stats["running"] == 0


def test_serve_admission_respects_memory_budget(rbf):
    """A budget that holds one request at a time: the requests run one after
    the other (no two admitted intervals overlap) although four slots are free,
    and the slots' charged bytes never exceed the budget."""
    reqs = requests(rbf, [(96, 0.9, False), (100, 0.9, False), (90, 0.95, False), (80, 1.0, False)], seed=400)
    fps = []
    for p, cfg in reqs:
        w = np.zeros(p.n)
        fps.append(rbf.rbf_request_footprint(rbf.make_request(p.xy, p.f, w, cfg)))
    budget = int(1.6 * max(fps))
    srv = rbf.Server(0, slots=4, mem_budget=budget)
    tickets = [srv.submit(p.xy, p.f, cfg) for p, cfg in reqs]
    results = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    spans = sorted((r.t_admit, r.t_done) for _, r, _ in results)
    for a, b in zip(spans, spans[1:]):
        assert b[0] >= a[1]
    assert stats["peak_resident_bytes"] <= budget
    for (p, cfg), (_, r, w) in zip(reqs, results):
        assert r.status == 0
        _, wa = alone(rbf, p, cfg)
        np.testing.assert_array_equal(w, wa)
        assert oracle_relres(p, w) <= 1e-13


def test_serve_rejects_request_over_budget(rbf):
    (p, cfg), = requests(rbf, [(64, 0.9, False)])
    srv = rbf.Server(0, slots=2, mem_budget=1 << 20)
    with pytest.raises(rbf.RbfError) as e:
        srv.submit(p.xy, p.f, cfg)
    assert e.value.status == 2
    srv.close()


def test_serve_wait_timeout_then_result(rbf):
    (p, cfg), = requests(rbf, [(512, 0.8, True)], seed=500)
    srv = rbf.Server(0, slots=1)
    t = srv.submit(p.xy, p.f, cfg)
    st, _, w = srv.wait(t, 0.0)
    assert st == 7 and w is None
    st, r, w = srv.wait(t)
    assert st == 0 and r.status == 0 and r.info.relres <= 1e-13
    st2, _, _ = srv.wait(t)
    assert st2 == 1   # the ticket is forgotten once collected
    srv.close()


def test_serve_destroy_with_queued_requests(rbf):
    reqs = requests(rbf, [(64, 0.9, True)] * 4, seed=600)
    srv = rbf.Server(0, slots=1)
    for p, cfg in reqs:
        srv.submit(p.xy, p.f, cfg)
    srv.close()   # the running request finishes, the queued ones are failed; returns
