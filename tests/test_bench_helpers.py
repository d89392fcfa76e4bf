"""bench.py's roofline objects on CPU: the fields the JSON line must carry,
frac = achieved / peak, and ceilings that follow from the issue rate and the
per-revision instruction counts."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_issue_peak_from_unit_counts():
    assert bench.ISSUE_PEAK_LANE_INSTR == pytest.approx(152 * 4 * 32 * 2.07e9)


def test_f64_roofline_object():
    pairs, avg_s = 375_552_506, 2.27e-3
    r = bench.f64_matvec_roofline(pairs, avg_s, 185, traffic=True)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r
    assert r["bound"] == "alu" and r["unit"] == "Gpair/s"
    assert r["achieved"] == pytest.approx(pairs / avg_s / 1e9)
    instr = bench.MATVEC_F64_INSTR_PER_PAIR[bench.MATVEC_F64_REV]
    assert r["peak"] == pytest.approx(bench.ISSUE_PEAK_LANE_INSTR / instr / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == bench.MATVEC_F64_TRAFFIC[bench.MATVEC_F64_REV]
    assert r["kernel_rev"] == bench.MATVEC_F64_REV
    # traffic is only claimed for the workload the counters were taken on
    assert bench.f64_matvec_roofline(pairs, avg_s, 185, traffic=False)["traffic"] is None


def test_roofline_constants_are_per_revision():
    assert bench.MATVEC_F64_REV in bench.MATVEC_F64_INSTR_PER_PAIR
    assert bench.MATVEC_F64_REV in bench.MATVEC_F64_TRAFFIC
    # algorithmic bytes of the FP64 matvec are 32 B per point; the measured traffic sits above them
    assert bench.MATVEC_F64_TRAFFIC[bench.MATVEC_F64_REV] >= 32 * 1024 * 1024
    assert 4.0 < bench.MATVEC_F32_INSTR_PER_CANDIDATE < 10.0
    assert bench.MATVEC_F32_TRAFFIC > 0


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
