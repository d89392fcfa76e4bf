"""bench.py's roofline objects on CPU: the fields the JSON line must carry,
frac = achieved / peak, and ceilings that follow from unit counts and clocks
alone (no per-revision instruction counts)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_peaks_from_unit_counts():
    assert bench.ISSUE_PEAK_LANE_INSTR == pytest.approx(152 * 4 * 32 * 2.07e9)
    assert bench.FP64_DFMA_PEAK_PAIRS == pytest.approx(152 * 2 * 2.07e9)      # 629.3 G pairs/s
    assert bench.MUFU_PEAK_PAIRS == pytest.approx(152 * 16 * 2.07e9)          # 5.03 T pairs/s


def test_f64_roofline_object():
    pairs, avg_s = 375_552_506, 2.27e-3
    r = bench.f64_matvec_roofline(pairs, avg_s, 185, 37_978_112)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r
    assert r["bound"] == "alu" and r["unit"] == "Gpair/s"
    assert r["achieved"] == pytest.approx(pairs / avg_s / 1e9)
    assert r["peak"] == pytest.approx(629.28, rel=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    ib = r["issue_bound"]
    assert ib["peak"] == pytest.approx(bench.ISSUE_PEAK_LANE_INSTR / bench.F64_ISSUE_BUDGET_PER_PAIR / 1e9)
    assert ib["frac"] == pytest.approx(r["achieved"] / ib["peak"])
    assert r["traffic"] == 37_978_112
    assert bench.f64_matvec_roofline(pairs, avg_s, 185, None)["traffic"] is None


def test_f64_replay_roofline_takes_the_larger_bound():
    """The replay's two bounds: bytes over the measured copy bandwidth and one
    DFMA per pair; the slower one is the object's bound, the other beside it."""
    hbm, _ = bench.hbm_peak_gbs()
    pairs, n = 18_543_323_276, 51_380_224
    dfma_s = pairs / bench.FP64_DFMA_PEAK_PAIRS
    # bytes that take exactly twice the DFMA time: HBM-bound at half speed
    store = int(2 * dfma_s * hbm * 1e9) - 16 * n
    r = bench.f64_replay_roofline(pairs, n, store, 4 * dfma_s, 7)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
    assert abs(r["frac"] - 0.5) < 1e-9
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9
    assert r["other_bound"]["bound"] == "alu" and abs(r["other_bound"]["frac"] - 0.25) < 1e-9
    assert r["algorithmic_bytes_per_launch"] == store + 16 * n
    # the measured traffic, scaled by pairs: at least the 8 B value of each pair
    t_cap, pairs_cap = bench.MATVEC_F64_REPLAY_TRAFFIC[bench.MATVEC_F64_REPLAY_REV]
    assert t_cap >= 8 * pairs_cap
    assert abs(r["traffic"] - t_cap * pairs / pairs_cap) < 1.0
    # few bytes: the FP64 pipe bounds it
    r = bench.f64_replay_roofline(pairs, n, 8 * n, 2 * dfma_s, 7)
    assert r["bound"] == "alu" and abs(r["frac"] - 0.5) < 1e-9 and r["other_bound"]["bound"] == "hbm"


def test_f32_roofline_counts_in_cutoff_pairs_not_candidates():
    pairs, cand, avg_s = 191_000_000, 542_600_000, 127e-6
    r = bench.f32_matvec_roofline(pairs, cand, avg_s, 180, None, "inner")
    assert r["unit"] == "Tpair/s" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(pairs / avg_s / 1e12)
    assert r["frac"] == pytest.approx(pairs / avg_s / bench.MUFU_PEAK_PAIRS)
    assert r["stencil_candidates_per_pair"] == pytest.approx(cand / pairs)
    assert r["kernel"] == bench.MATVEC_F32_KERNEL and r["kernel_rev"] == bench.MATVEC_F32_REV


def test_f32_traffic_constant_is_for_the_current_revision():
    t, n = bench.MATVEC_F32_TRAFFIC[bench.MATVEC_F32_REV]
    assert t >= 16 * n   # at least the algorithmic 16 B per point (offsets 8, w 4, y 4)


def test_roofline_constants():
    assert bench.MATVEC_F64_REV in bench.MATVEC_F64_TRAFFIC
    # algorithmic bytes of the FP64 matvec are 32 B per point; the measured traffic sits above them
    assert bench.MATVEC_F64_TRAFFIC[bench.MATVEC_F64_REV] >= 32 * 1024 * 1024
    assert 60.0 < bench.F64_ISSUE_BUDGET_PER_PAIR < 160.0


def test_lattice_window_is_a_block_of_the_lattice():
    p = bench.W.lattice_problem(40, 0.8, seed=3)
    xy, f, x0, y0, (i0, j0, w) = bench.lattice_window(p, 16, seed=5)
    assert w == 16 and i0 % 4 == 0 and j0 % 4 == 0
    full = p.xy.reshape(40, 40, 2)
    np = bench.np
    assert np.array_equal(xy.reshape(16, 16, 2), full[j0:j0 + 16, i0:i0 + 16])
    assert np.array_equal(f, p.f.reshape(40, 40)[j0:j0 + 16, i0:i0 + 16].ravel())
    # the window's box origin lies on the full lattice's box edges
    assert x0 == pytest.approx(p.x0 + i0 * p.h) and y0 == pytest.approx(p.x0 + j0 * p.h)
    assert bench.lattice_window(p, 100, seed=1)[4] == (0, 0, 40)


def test_every_workload_has_a_description():
    for name, (_, desc) in bench.WORKLOADS.items():
        assert isinstance(desc, str) and len(desc) > 10, name


@pytest.mark.timeout(600)
def test_reference_arm_json_line_on_the_small_lattice():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON
    line with the contract's keys; it needs no GPU."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "lattice64", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "lattice64"
    # ms_per_step is the wall time of the step's sample, which fits in the run
    assert 0.0 < line["ms_per_step"] < 600e3
