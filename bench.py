"""Benchmark: time of one Gaussian RBF interpolation solve to relative residual
1e-13 (GMRES(30) + RASM, cell-list truncated matvec) on a GB300, mixed
precision (FP32 inner GMRES, FP64 refinement) against the plain FP64 form on
the same inputs, with a short serving run's p50 / p99 latency in the same line.

One step = the whole path on one problem: cell binning, subdomain lists and
RASM factors, and the GMRES solve (every row of the hot path), inputs resident
in HBM when the step starts. L2 is flushed (a 256 MB write) before every timed
step; the step's working set (Krylov basis, subdomain inverses) is itself
many times L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lattice7168|lattice1024|lattice64|batch4096|serve|paper]
                    [--mode mixed|f64]

Default: the 7168 x 7168 jittered lattice (N = 51,380,224), mixed precision.

With --gpus N > 1 (launched by torchrun) each rank solves its own replica of
the problem ("replicas only": the problems are independent), times are the
max over ranks, and value stays the time per solve.

--impl reference times the CPU oracle (plain FP64 C, OpenMP) on the host
cores: every step solves part of a window of the same lattice (setup, one
matvec, one RASM apply, a few GMRES steps) and projects the full solve per
point and per iteration (see cpu_baseline.sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0909_5413_gb300 import workloads as W  # noqa: E402

METRIC = "RBF solve time at 1e-13 rel. residual (GMRES+RASM), mixed vs FP64; serve p50/p99"
UNIT = "ms"

SM_COUNT, SM_CLOCK_HZ = 152, 2.07e9

# FP64 matvec roofline. Every in-cutoff pair needs one FP64 FMA (the
# accumulate of k_ij w_j; the kernel value itself is integer work on the
# fixed-point path), and GB300 issues 2 DFMA per SM per clock: the FP64-pipe
# bound is 152 x 2 x 2.07 GHz = 629.3 G pairs/s, fixed by the algorithm.
# Second bound, the SM's instruction issue (152 x 4 x 32 lanes x 2.07 GHz =
# 40.3 T lane-instructions/s) over the fixed-point algorithm's own
# instruction budget per in-cutoff pair: 66 32-bit operations for the pair
# offset, the squares, the multiply-high by the exponent scale, the two table
# products, the remainder polynomial and the FP64 assembly; 7 for walking the
# accepted-source mask (bit scan, clear, index, two coordinate loads); and the
# packed FP32 cutoff filter, 6.5 per candidate over 9/pi = 2.86 candidates per
# pair of the 3 x 3 stencil of r_c cells: 92 per pair, 438 G pairs/s. Both
# are counted from the algorithm once and do not follow a kernel revision.
FP64_DFMA_PEAK_PAIRS = SM_COUNT * 2 * SM_CLOCK_HZ
ISSUE_PEAK_LANE_INSTR = SM_COUNT * 4 * 32 * SM_CLOCK_HZ
F64_ISSUE_BUDGET_PER_PAIR = 92.0
MATVEC_F64_REV = "fixed-point-v6"
# DRAM read + write of one launch on the 1024 x 1024 lattice (ncu, this revision)
MATVEC_F64_TRAFFIC = {"fixed-point-v5": 37_978_112, "fixed-point-v6": 38_016_427}
FLOPS_PER_PAIR_F64 = 26   # FP64-equivalent flops of one pair (dx, dy 2; r2 3; argument 1; exp 18; accumulate 2)
# The replay of kept pair values (RBF_OPT_STORE_F64) reads, per launch, the
# values and masks (rbf_store_f64_bytes) plus w and y (16 B per point), and
# issues one DFMA per pair: bound by the larger of the two times.
MATVEC_F64_REPLAY_REV = "replay-v3"
# DRAM read + write of one replay on the 1024 x 1024 lattice (ncu, this revision) and the
# in-cutoff pairs it replayed: scaled to another workload by its pairs
MATVEC_F64_REPLAY_TRAFFIC = {"replay-v3": (3_378_374_981, 375_552_506)}


def hbm_peak_gbs() -> tuple[float, str]:
    """The measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def f64_replay_roofline(pairs: int, n: int, store_bytes: int, avg_s: float, launches: int, note: str = "") -> dict:
    """Roofline object of the FP64 replay: the HBM bytes it must read and write
    against the measured copy bandwidth, and its DFMAs against the FP64 pipe."""
    hbm_gbs, src = hbm_peak_gbs()
    nbytes = store_bytes + 16 * n
    t_hbm = nbytes / (hbm_gbs * 1e9)
    t_dfma = pairs / FP64_DFMA_PEAK_PAIRS
    hbm = {"bound": "hbm", "achieved": nbytes / avg_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
           "frac": t_hbm / avg_s, "peak_note": f"copy bandwidth, {src}"}
    alu = {"bound": "alu", "achieved": pairs / avg_s / 1e9, "peak": FP64_DFMA_PEAK_PAIRS / 1e9, "unit": "Gpair/s",
           "frac": t_dfma / avg_s,
           "peak_note": "FP64 pipe: one DFMA per in-cutoff pair, 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    main, other = (hbm, alu) if t_hbm >= t_dfma else (alu, hbm)
    traffic = None
    if MATVEC_F64_REPLAY_REV in MATVEC_F64_REPLAY_TRAFFIC:
        t_cap, pairs_cap = MATVEC_F64_REPLAY_TRAFFIC[MATVEC_F64_REPLAY_REV]
        traffic = t_cap * pairs / pairs_cap
    out = {"kernel": "k_matvec_f64 (replay of the kept pair values)", **main, "traffic": traffic,
           "other_bound": other, "kernel_rev": MATVEC_F64_REPLAY_REV, "pairs_per_launch": pairs,
           "algorithmic_bytes_per_launch": nbytes, "store_bytes": store_bytes,
           "store_bytes_per_pair": store_bytes / pairs, "avg_launch_ms": avg_s * 1e3, "launches": launches}
    if traffic is not None:
        out["traffic_note"] = ("ncu DRAM read + write of one replay on the 1024 x 1024 lattice (3.378 GB, "
                               "1.00x its algorithmic bytes) x in-cutoff pairs / 375,552,506")
    if note:
        out["note"] = note
    return out


def f64_matvec_roofline(pairs: int, avg_s: float, launches: int, traffic, note: str = "") -> dict:
    """Roofline object of the FP64 matvec from its in-cutoff pair count and
    CUDA-event launch time, against the FP64-pipe bound (one DFMA per pair)."""
    rate = pairs / avg_s
    issue_peak = ISSUE_PEAK_LANE_INSTR / F64_ISSUE_BUDGET_PER_PAIR
    out = {"kernel": "k_matvec_f64", "bound": "alu", "achieved": rate / 1e9, "peak": FP64_DFMA_PEAK_PAIRS / 1e9,
           "unit": "Gpair/s", "frac": rate / FP64_DFMA_PEAK_PAIRS, "traffic": traffic,
           "peak_note": ("FP64 pipe: one DFMA per in-cutoff pair, 152 SMs x 2 DFMA/clk x 2.07 GHz "
                         "(derived from unit counts and clocks; no FP64 figure is measured)"),
           "issue_bound": {"budget_lane_instr_per_pair": F64_ISSUE_BUDGET_PER_PAIR, "peak": issue_peak / 1e9,
                           "frac": rate / issue_peak},
           "kernel_rev": MATVEC_F64_REV, "pairs_per_launch": pairs, "avg_launch_ms": avg_s * 1e3,
           "launches": launches,
           "fp64_equivalent": {"tflops": pairs * FLOPS_PER_PAIR_F64 / avg_s / 1e12,
                               "fp64_peak_tflops": FP64_DFMA_PEAK_PAIRS * 2 / 1e12,
                               "flops_per_pair": FLOPS_PER_PAIR_F64}}
    if note:
        out["note"] = note
    return out


# FP32 matvec roofline (the inner solves of the mixed form). Every in-cutoff
# pair at the inner cutoff needs one exp2 on the SFU (MUFU.EX2), which issues
# 16 results per SM per clock: 152 x 16 x 2.07 GHz = 5.03 T pairs/s. The
# symmetric kernel evaluates each neighbouring cell pair once, every pair of
# the two cells (no mask), so its useful rate is in-cutoff pairs
# (rbf_count_pairs on the inner grid) over the launch time (the symmetric
# kernel and its gather); the 3 x 3 stencil's candidate count is reported
# beside it.
MUFU_PEAK_PAIRS = SM_COUNT * 16 * SM_CLOCK_HZ
MATVEC_F32_REV = "sym-colsum-v4"
MATVEC_F32_KERNEL = "k_matvec_f32_sym<TPL> + k_sym_gather"
# DRAM read + write of one launch on the 7168 x 7168 lattice's inner grid
# (ncu, one-pass dram__bytes metrics, this revision): the symmetric kernel of
# the 33-64 point cells 630.8 MB + 976.9 MB (its five FP32 slots per point
# written), the gather 1230 MB + 192.3 MB; and that lattice's N
MATVEC_F32_TRAFFIC = {"sym-colsum-v4": (3_030_010_000, 51_380_224)}


def f32_matvec_roofline(pairs: int, cand: int, avg_s: float, launches: int, traffic, grid: str) -> dict:
    rate = pairs / avg_s
    return {"kernel": MATVEC_F32_KERNEL, "bound": "alu", "achieved": rate / 1e12, "peak": MUFU_PEAK_PAIRS / 1e12,
            "unit": "Tpair/s", "frac": rate / MUFU_PEAK_PAIRS, "traffic": traffic,
            "peak_note": ("SFU: one ex2 per in-cutoff pair at the inner cutoff, 152 SMs x 16 MUFU.EX2/clk x 2.07 GHz "
                          "(derived from unit counts and clocks)"),
            "kernel_rev": MATVEC_F32_REV, "pairs_per_launch": pairs, "stencil_candidates_per_launch": cand,
            "stencil_candidates_per_pair": cand / max(pairs, 1),
            "avg_launch_ms": avg_s * 1e3, "launches": launches, "grid": grid}


WORKLOADS = {
    "lattice64": (W.config_small, "64x64 jittered lattice on [-1,1]^2 (N=4,096)"),
    "lattice1024": (W.config_1m, "1024x1024 jittered lattice on [-1,1]^2 (N=1,048,576)"),
    "lattice2048": (W.config_4m, "2048x2048 jittered lattice on [-1,1]^2 (N=4,194,304)"),
    "lattice7168": (W.config_51m, "7168x7168 jittered lattice on [-1,1]^2 (N=51,380,224)"),
    "batch4096": (None, "independent jittered lattices on [-1,1]^2, N log-uniform in [256, 16384], "
                        "h/sigma uniform in [0.6, 1.0], f = sum of four random Gaussians, one seed per problem"),
    "serve": (None, "requests with Poisson arrivals, N log-uniform in [1e3, 4e6] (jittered lattices on [-1,1]^2), "
                    "h/sigma uniform in [0.6, 1.0], f = sum of four random Gaussians"),
    "paper": (None, "Franke's function on a lattice over [0,1]^2, sigma = 0.001 (N about 1.0e6 to 1.6e6), "
                    "subdomains B = 5 sigma, D = 1.9 B, h/sigma in {0.8, 0.9, 1.0}; RASM and ASM; "
                    "interpolant evaluated onto a 2048 x 2048 lattice"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lattice7168", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default=None, choices=["f64", "mixed"],
                    help="precision of the timed form (default mixed; the other is measured beside it)")
    ap.add_argument("--batch-count", type=int, default=4096, help="problems of the batch workload")
    ap.add_argument("--max-iters", type=int, default=3000, help="GMRES step cap per problem (batch, serve)")
    ap.add_argument("--requests", type=int, default=64, help="requests of the serve workload")
    ap.add_argument("--slots", type=int, default=8, help="server slots (serve)")
    ap.add_argument("--rates", default="0.5,0.9", help="arrival rates swept, as fractions of the saturated rate")
    ap.add_argument("--sigma", type=float, default=0.001, help="Gaussian width of the paper workload")
    ap.add_argument("--inner-cutoff", type=float, default=6.1,
                    help="mixed form: cutoff (in sigma) of the FP32 inner grid; 0 = the r_c grid")
    ap.add_argument("--tune", action="store_true",
                    help="autotune the cell size and matvec tiles (rbf_tune) once, before the warm-up steps")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other-precision measurement")
    ap.add_argument("--no-store", action="store_true",
                    help="keep no FP64 pair values: every FP64 product evaluates its pairs")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving run of a single-problem line")
    ap.add_argument("--serve-requests", type=int, default=16, help="requests of the short serving run")
    ap.add_argument("--window", type=int, default=0,
                    help="lattice side of the oracle's window sample (0: 2048 for the CPU baseline, 1024 per "
                         "reference step)")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of the ranks' values (the slowest replica sets the time);
    the value itself when there is one rank (dist is None)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(name: str, p, mode: str, inner_cutoff: float | None = None) -> dict:
    return {"workload": name, "description": WORKLOADS[name][1], "n_points": p.n,
            "h_over_sigma": round(p.h / p.sigma, 6), "cutoff_sigmas": 8.6,
            "rasm": "4x4 lattice-point cores + 1-point ring", "gmres_restart": 30, "rtol": 1e-13,
            "precision": mode, "inner_cutoff_sigmas": inner_cutoff if mode == "mixed" else None,
            "l2": "flushed (256 MB write) before each timed step", "parallelism": "replicas"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # raw samples: RBF_BENCH_LOG_DIR if set, else the system temporary directory
        log_dir = os.environ.get("RBF_BENCH_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle

def lattice_window(p, win: int, seed: int):
    """A win x win window of the problem's lattice (the same points, in user
    order), at a seeded offset aligned to the 4 x 4-point subdomain cores, with
    its own subdomain box origin on the same box edges as the full lattice."""
    n = p.n_side
    win = min(win, n)
    rng = np.random.default_rng(seed)
    i0 = 4 * int(rng.integers(0, (n - win) // 4 + 1))
    j0 = 4 * int(rng.integers(0, (n - win) // 4 + 1))
    xy = np.ascontiguousarray(p.xy.reshape(n, n, 2)[j0:j0 + win, i0:i0 + win].reshape(-1, 2))
    f = np.ascontiguousarray(p.f.reshape(n, n)[j0:j0 + win, i0:i0 + win].reshape(-1))
    return xy, f, p.x0 + i0 * p.h, p.x0 + j0 * p.h, (i0, j0, win)


def oracle_window_sample(p, win: int, seed: int, counts: dict, sample_steps: int = 6) -> dict:
    """The CPU oracle on a window of the workload's lattice: setup (binning,
    lists, subdomain factors), one FP64 matvec, one RASM apply and
    sample_steps GMRES steps, timed; projected to the full problem per point
    (every part of the method is O(N)) and per iteration with the given
    counts (iterations and restart cycles of an FP64 solve of the full
    problem). When the window is the whole lattice and counts are None the
    solve runs to the end instead and is timed as it stands."""
    from oracle import oracle as O

    threads = os.cpu_count() or 1
    O.set_threads(threads)
    xy, f, x0, y0, (i0, j0, w) = lattice_window(p, win, seed)
    t_wall = time.perf_counter()
    t0 = time.perf_counter()
    pr = O.Problem(xy, p.sigma, p.cutoff, x0, y0, p.core_size, p.overlap)
    t_setup = time.perf_counter() - t0
    if counts is None and w == p.n_side:
        t0 = time.perf_counter()
        _, info = pr.solve(f)
        t_solve = time.perf_counter() - t0
        pr.close()
        return {"value": (t_setup + t_solve) * 1e3, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": (f"the whole workload, N={p.n}: oracle setup ({t_setup:.2f} s) and FP64 GMRES+RASM solve "
                           f"({info.iters} steps, relres {info.relres:.2e}, {t_solve:.2f} s), end to end"),
                "measured_s": round(time.perf_counter() - t_wall, 3), "iters": info.iters}
    t0 = time.perf_counter()
    pr.matvec(f)
    t_mv = time.perf_counter() - t0
    t0 = time.perf_counter()
    pr.rasm_apply(f)
    t_ap = time.perf_counter() - t0
    t0 = time.perf_counter()
    pr.solve(f, max_iters=sample_steps)
    t_s = time.perf_counter() - t0
    pr.close()
    # the sample ran: 2 true-residual matvecs, sample_steps x (apply + matvec + ortho), 1 final apply
    t_ortho = max(0.0, (t_s - (sample_steps + 2) * t_mv - (sample_steps + 1) * t_ap) / sample_steps)
    iters, cycles = counts["iters"], counts["restarts"]
    scale = p.n / (w * w)
    proj = scale * (t_setup + (iters + cycles + 1) * t_mv + (iters + cycles) * t_ap + iters * t_ortho)
    return {"value": proj * 1e3, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"extrapolated per point and per iteration: a {w} x {w} window (N={w * w}, offset {i0}, {j0}) "
                       f"of the {p.n_side} x {p.n_side} lattice; oracle setup {t_setup:.2f} s, one FP64 matvec "
                       f"{t_mv:.3f} s, one RASM apply {t_ap:.3f} s, {sample_steps} GMRES steps {t_s:.2f} s; "
                       f"scaled by N / N_window = {scale:.2f} to {iters} steps in {cycles} cycles ({counts['source']})"),
            "measured_s": round(time.perf_counter() - t_wall, 3)}


def run_reference(args, ws, rank):
    """Reference arm: the oracle as it stands on the host cores. Each step is a
    bounded sample (a seeded window of the lattice, setup + matvec + apply +
    six GMRES steps) projected to the full solve; ms_per_step is the wall time
    of those samples, value the projected solve time."""
    if rank != 0:
        return
    name = args.workload
    p = WORKLOADS[name][0]()
    from oracle import oracle as O
    # iteration counts: the oracle's own full FP64 solve of a 512 x 512 window
    # (iteration counts do not depend on N, Sec. 3.2), untimed
    O.set_threads(os.cpu_count() or 1)
    xw, fw, x0, y0, _ = lattice_window(p, 512, seed=1)
    prw = O.Problem(xw, p.sigma, p.cutoff, x0, y0, p.core_size, p.overlap)
    _, winfo = prw.solve(fw)
    prw.close()
    counts = {"iters": winfo.iters, "restarts": winfo.restarts,
              "source": f"the oracle's own full solve of a {min(512, p.n_side)}-point-wide window"}
    win = args.window or 1024
    proj, wall = [], []
    cb = None
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = oracle_window_sample(p, win, seed=100 + step, counts=counts)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            proj.append(cb["value"])
            wall.append(dt * 1e3)
    v = statistics.mean(proj)
    cb["value"] = v
    cb["sample"] += f"; one seeded window per step, {args.steps} timed steps"
    mode = args.mode or "mixed"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(wall),
           "ms_per_step_is": "wall time of one step's oracle sample (value is the full solve it projects)",
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(name, p, mode, args.inner_cutoff), "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- GPU path

def short_serve(rbf, args, local) -> dict:
    """A short serving run for the single-problem line: serve-workload requests
    (N log-uniform in [1e3, 4e6]), a saturated burst, then Poisson arrivals at
    half the saturated rate; p50 / p99 latency of the Poisson run."""
    probs = W.batch_workload(args.serve_requests, lo=1000, hi=4_000_000, seed=W.DEFAULT_SEED + 5000)
    res = serve_sweep(rbf, args, local, probs, rates=[0.5], warm=1)
    row = res["rates"][0]
    return {"requests": len(probs), "n_points_total": int(sum(p.n for p in probs)), "slots": args.slots,
            "rate_frac": 0.5, "rate_per_s": row["rate_per_s"], "p50_ms": row["p50_ms"], "p99_ms": row["p99_ms"],
            "mean_ms": row["mean_ms"], "throughput_per_s": row["throughput_per_s"],
            "saturated": res["saturated"], "converged": row["converged"],
            "relres_max_converged": res["solve"]["relres_max_converged"],
            "note": "mixed precision, inner cutoff 6.1 sigma; requests with h/sigma < 0.7 stop on stagnation"}


def timed_steps(fn, reps, flush, barrier):
    import torch
    ts, last = [], None
    for _ in range(reps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        last = fn()
        e1.record()
        barrier()
        ts.append(e0.elapsed_time(e1))
    return ts, last


def run_ours(args, ws, rank, local):
    import torch

    from paper_0909_5413_gb300 import rbf

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = args.workload
    p = WORKLOADS[name][0]()
    mode = args.mode or "mixed"

    def cfg_for(md):
        return rbf.config_for(p, mixed=(md == "mixed"), factor_precision=rbf.RBF_FP32 if md == "mixed" else rbf.RBF_FP64,
                              inner_cutoff=args.inner_cutoff if md == "mixed" else 0.0)
    cfg = cfg_for(mode)
    xy = torch.from_numpy(p.xy).cuda()
    f = torch.from_numpy(p.f).cuda()
    w = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ctx = rbf.Context(local)
    h = ctx.handle
    if args.no_store:   # every FP64 product evaluates its pairs (nothing kept)
        rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, 0)

    def step(c):
        w.zero_()
        ctx.bin(xy, c)
        ctx.rasm_setup(c)
        st, info = ctx.solve(f, w, c, check=False)
        return st, info

    tuned = None
    if args.tune:
        # one FP64 matvec per step for the FP64 form; about 1 FP64 per 26 FP32 ones for the mixed form
        best, score = rbf.rbf_tune(h, xy, p.n, cfg.params(), 1.0, 26.0 if mode == "mixed" else 0.0)
        cfg.cell_size, cfg.tile_f64, cfg.tile_f32 = best.cell_size, best.tile_f64, best.tile_f32
        tuned = {"cell_size_over_rc": best.cell_size / p.cutoff, "tile_f64": best.tile_f64,
                 "tile_f32": best.tile_f32, "score_ms": score}

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        step(cfg)
    torch.cuda.synchronize()
    # inside the timed region only the dominant kernel's launches carry event
    # records (its live duration for the roofline); the per-class breakdown
    # comes from one extra profiled step after the timed region
    dominant = rbf.RBF_PROF_MATVEC_F64 if mode == "f64" else rbf.RBF_PROF_MATVEC_F32
    rbf.rbf_profile_classes(h, 1 << dominant)
    rbf.rbf_profile_enable(h, True)
    for k in range(rbf.RBF_PROF_COUNT):
        rbf.rbf_profile_read(h, k)   # discard warm-up records
    launches0 = ctx.launches
    clocks = ClockSampler(local)
    clocks.start()
    times, outs = [], []
    for _ in range(args.steps):
        ts, r = timed_steps(lambda: step(cfg), 1, flush, barrier)
        times += ts
        outs.append(r)
    clk = clocks.stop()
    launches = ctx.launches - launches0
    prof = {k: rbf.rbf_profile_read(h, k) for k in range(rbf.RBF_PROF_COUNT)}
    rbf.rbf_profile_classes(h, 0xFFFFFFFF)
    flush.zero_()
    step(cfg)                             # the breakdown step (untimed, every class recorded)
    torch.cuda.synchronize()
    prof_all = {k: rbf.rbf_profile_read(h, k) for k in range(rbf.RBF_PROF_COUNT)}
    rbf.rbf_profile_enable(h, False)
    ms = max_over_ranks(statistics.mean(times), dist, "cuda")
    stats = [st for st, _ in outs]
    info = outs[-1][1].as_dict()
    ok = all(s == 0 for s in stats) and info["relres"] <= 1e-13

    # dominant kernel: the truncated matvec of the timed precision
    roofline, roof64 = None, None
    pairs = rbf.rbf_count_neighbors(h)
    store_bytes = rbf.rbf_store_f64_bytes(h)   # the FP64 products replayed kept values
    n_mv, t_mv = prof[dominant]
    if n_mv and mode == "mixed":
        inner = args.inner_cutoff > 0
        pairs_in = rbf.rbf_count_pairs(h, 1 if inner else 0)
        cand = rbf.rbf_count_candidates(h, 1 if inner else 0)
        traffic = None
        if inner and args.inner_cutoff == 6.1 and not args.tune and MATVEC_F32_REV in MATVEC_F32_TRAFFIC:
            # the 7168 x 7168 capture, scaled by the points processed
            t_cap, n_cap = MATVEC_F32_TRAFFIC[MATVEC_F32_REV]
            traffic = t_cap * p.n / n_cap
        roofline = f32_matvec_roofline(pairs_in, cand, t_mv / n_mv / 1e3, n_mv, traffic,
                                       f"inner, cells of {args.inner_cutoff} sigma" if inner else "cells of side r_c")
        if traffic is not None:
            roofline["traffic_note"] = ("ncu DRAM read + write of one launch (symmetric kernel and gather) on the "
                                        "7168 x 7168 lattice x N / 51,380,224; algorithmic 16 B per point plus "
                                        "40 B per point of slots")
    elif n_mv and store_bytes:
        roofline = f64_replay_roofline(pairs, p.n, store_bytes, t_mv / n_mv / 1e3, n_mv)
    elif n_mv:
        default_cfg = (cfg.cell_size in (0.0, p.cutoff)) and cfg.tile_f64 in (0, 128)
        traffic = MATVEC_F64_TRAFFIC.get(MATVEC_F64_REV) if default_cfg else None
        if traffic is not None:
            traffic = traffic * p.n / 1048576.0
        roofline = f64_matvec_roofline(pairs, t_mv / n_mv / 1e3, n_mv, traffic)
        if traffic is not None:
            roofline["traffic_note"] = ("ncu DRAM read + write of one launch on the 1024 x 1024 lattice x "
                                        "N / 1,048,576")
    # the FP64 matvec (outer residuals of the mixed form) from the breakdown step
    n64, t64 = prof_all[rbf.RBF_PROF_MATVEC_F64]
    if mode == "mixed" and n64:
        note = "outer FP64 residuals of the mixed solve, from the breakdown step"
        if store_bytes:
            roof64 = f64_replay_roofline(pairs, p.n, store_bytes, t64 / n64 / 1e3, n64, note=note)
        else:
            roof64 = f64_matvec_roofline(pairs, t64 / n64 / 1e3, n64, None, note=note)
    breakdown = {nm: {"launches": prof_all[k][0], "ms": round(prof_all[k][1], 3)} for nm, k in
                 (("matvec_f64", 0), ("matvec_f32", 1), ("rasm_apply", 2), ("orthogonalisation", 3),
                  ("rasm_setup", 4), ("binning", 5), ("fp64_values_kept", 6))}
    tc, f64 = rbf.rbf_rasm_factor_counts(h)
    factors = {"precision": "fp32 tensor cores" if mode == "mixed" else "fp64", "tensor_core_subdomains": tc,
               "fp64_subdomains": f64}

    # end to end through the host-buffer entry point, right after the timed
    # steps (before the other forms below change the context's state)
    e2e = None
    if not args.no_e2e:
        xy_h = torch.from_numpy(p.xy.copy()).pin_memory()
        f_h = torch.from_numpy(p.f.copy()).pin_memory()
        w_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
        ctx.interpolate_host(xy_h, f_h, w_h, cfg, check=False)
        te, _ = timed_steps(lambda: ctx.interpolate_host(xy_h, f_h, w_h, cfg, check=False),
                            max(1, min(args.steps, 3)), flush, barrier)
        e2e = {"value": max_over_ranks(statistics.mean(te), dist, "cuda"), "unit": UNIT,
               "h2d_bytes_per_step": xy_h.numel() * 8 + f_h.numel() * 8, "d2h_bytes_per_step": w_h.numel() * 8,
               "call": "rbf_interpolate_host (pinned host buffers, copies inside the timed region)"}
        del xy_h, f_h, w_h

    # the mixed form with subdomain inverses computed in FP64 (stored FP32), for
    # the inner-step cost of the tensor-core inverses
    if mode == "mixed" and not args.no_extra:
        c3 = cfg_for("mixed")
        c3.factor_precision = rbf.RBF_FP32_FROM_FP64
        flush.zero_()
        step(c3)
        ts, (st3, i3) = timed_steps(lambda: step(c3), 1, flush, barrier)
        factors["fp64_computed_inverses"] = {"ms_per_step": ts[0], "iters": i3.iters, "relres": i3.relres,
                                             "status": st3}
        factors["inner_step_ratio_tc_over_fp64"] = info["iters"] / max(i3.iters, 1)

    # the other precision on the same inputs, for the "mixed vs FP64" comparison
    extra = None
    if not args.no_extra:
        other = "f64" if mode == "mixed" else "mixed"
        c2 = cfg_for(other)
        flush.zero_()
        step(c2)
        ts, (st2, i2) = timed_steps(lambda: step(c2), max(1, min(args.steps, 3)), flush, barrier)
        extra = {"precision": other, "ms_per_step": max_over_ranks(statistics.mean(ts), dist, "cuda"),
                 "steps": len(ts), "step_ms": [round(t, 3) for t in ts], "status": st2, **i2.as_dict()}
        extra["speedup_mixed_over_f64"] = (extra["ms_per_step"] / ms) if mode == "mixed" else (ms / extra["ms_per_step"])

    ctx.close()
    del w, flush
    torch.cuda.empty_cache()

    serve = None
    if not args.no_serve:
        serve = short_serve(rbf, args, local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        f64_counts = extra if (extra and extra["precision"] == "f64") else (info if mode == "f64" else None)
        counts = None
        if f64_counts is not None:
            counts = {"iters": f64_counts["iters"], "restarts": f64_counts["restarts"],
                      "source": "the GPU's FP64 solve of the full problem"}
        if p.n <= 1100000:
            cpu = oracle_window_sample(p, p.n_side, seed=0, counts=None)
        else:
            if counts is None:
                counts = {"iters": info["iters"], "restarts": info["restarts"],
                          "source": "the GPU's mixed solve of the full problem (inner steps)"}
            cpu = oracle_window_sample(p, args.window or 2048, seed=0, counts=counts)

    if rank == 0:
        out = {"metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if mode == "f64" else "f32-inner/f64-outer", "data": "synthetic",
               "config": {**workload_config(name, p, mode, args.inner_cutoff), "tuned": tuned,
                          "fp64_products": "replay kept values" if store_bytes else "evaluated"},
               "value_is": f"{mode} solve (bin + RASM setup + GMRES) to relres 1e-13, mean of the timed steps",
               "ok": ok, "solve": info, "step_ms": [round(t, 3) for t in times], "roofline": roofline,
               "roofline_f64_matvec": roof64, "breakdown_ms": breakdown, "rasm_factors": factors,
               "breakdown_note": "one extra step after the timed region with every kernel class recorded",
               "other_precision": extra, "serve": serve, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clk}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------- many-problem batch

BATCH_METRIC = "RBF batch solve time at 1e-13 rel. residual (4096 independent problems, GMRES+RASM)"
RATIO_BINS = ((0.6, 0.7), (0.7, 0.8), (0.8, 0.9), (0.9, 1.0001))


def batch_problems(args):
    return W.batch_workload(args.batch_count)


def batch_config(args, probs, mode: str) -> dict:
    ns = np.array([p.n for p in probs])
    return {"workload": "batch4096" if args.batch_count == 4096 else f"batch{args.batch_count}",
            "description": WORKLOADS["batch4096"][1], "problems": len(probs), "n_points_total": int(ns.sum()),
            "n_min": int(ns.min()), "n_max": int(ns.max()), "cutoff_sigmas": 8.6,
            "rasm": "4x4 lattice-point cores + 1-point ring", "gmres_restart": 30, "rtol": 1e-13,
            "max_iters_per_problem": args.max_iters, "precision": mode,
            "inner_cutoff_sigmas": args.inner_cutoff if mode == "mixed" else None,
            "l2": "flushed (256 MB write) before each timed step", "parallelism": "replicas",
            "fp64_products": "evaluated" if args.no_store else "kept values replayed while every problem runs"}


def batch_summary(probs, infos, stats_w=None) -> dict:
    st = np.array([i.status for i in infos])
    stg = np.array([i.stagnated for i in infos])
    it = np.array([i.iters for i in infos])
    rr = np.array([i.relres for i in infos])
    ratio = np.array([p.h / p.sigma for p in probs])
    conv = st == 0
    bins = {}
    for lo, hi in RATIO_BINS:
        sel = (ratio >= lo) & (ratio < hi)
        bins[f"{lo:.1f}-{min(hi, 1.0):.1f}"] = {"problems": int(sel.sum()), "converged": int((conv & sel).sum()),
                                               "median_iters": float(np.median(it[sel & conv])) if (sel & conv).any()
                                               else None}
    return {"converged": int(conv.sum()), "stagnated": int(stg.sum()), "not_converged": int((~conv).sum()),
            "iters_median": float(np.median(it)), "iters_p90": float(np.percentile(it, 90)), "iters_max": int(it.max()),
            "relres_max_converged": float(rr[conv].max()) if conv.any() else None, "by_h_over_sigma": bins}


def oracle_batch_sample(probs, budget_s: float, seed: int, w_gpu=None, ptr=None, iters=None,
                        max_n: int | None = None) -> dict:
    """The CPU oracle on a seeded sample of the batch's problems, each solved on
    its own (setup and GMRES); problems are taken in a seeded random order until
    the budget is spent. With the GPU's per-problem step counts, each sampled
    solve runs that many steps and the time is projected to the whole batch by
    N x (steps + 1); otherwise each solve runs to 1e-13 (at most 3000 steps)
    and the projection is by N. With the GPU result, the sample also gives the
    relative error of w against the oracle's. Problems above max_n points are
    left out of the sample (the projection still covers them)."""
    from oracle import oracle as O

    threads = os.cpu_count() or 1
    O.set_threads(threads)
    order = np.random.default_rng(seed).permutation(len(probs))
    t_all, used, errs = 0.0, [], []
    for k in order:
        p = probs[k]
        if max_n is not None and p.n > max_n:
            continue
        mi = int(iters[k]) if iters is not None else 3000
        t0 = time.perf_counter()
        pr = O.Problem(p.xy, p.sigma, p.cutoff, p.x0, p.x0, p.core_size, p.overlap)
        wo, inf = pr.solve(p.f, max_iters=max(mi, 1))
        t_all += time.perf_counter() - t0
        used.append(int(k))
        if w_gpu is not None and inf.relres <= 1e-13:
            wg = w_gpu[ptr[k]:ptr[k + 1]]
            errs.append(float(np.linalg.norm(wg - wo) / np.linalg.norm(wo)))
        if t_all >= budget_s:
            break
    ns = np.array([p.n for p in probs], dtype=np.float64)
    wts = ns * (np.asarray(iters, dtype=np.float64) + 1.0) if iters is not None else ns
    proj = t_all * wts.sum() / wts[used].sum()
    out = {"value": proj * 1e3, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"{len(used)} of {len(probs)} problems (seeded random order) solved one by one by the oracle "
                      f"in {t_all:.2f} s" + (f" (problems of N <= {max_n} only)" if max_n else "") +
                      "; projected to all problems by " +
                      ("N x (GPU steps + 1)" if iters is not None else "N")),
           "measured_s": round(t_all, 3)}
    if errs:
        out["w_rel_error_vs_oracle_max"] = max(errs)
        out["w_rel_error_vs_oracle_problems"] = len(errs)
    return out


def run_reference_batch(args, ws, rank):
    if rank != 0:
        return
    probs = batch_problems(args)
    times, wall, cb = [], [], None
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = oracle_batch_sample(probs, budget_s=4.0, seed=step)
        if step >= args.warmup:
            times.append(cb["value"])
            wall.append((time.perf_counter() - t0) * 1e3)
    v = statistics.mean(times)
    cb["value"] = v
    out = {"impl": "reference", "metric": BATCH_METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(wall),
           "ms_per_step_is": "wall time of one step's oracle sample (value is the batch solve it projects)",
           "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": batch_config(args, probs, "f64"), "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args, ws, rank, local):
    import torch

    from paper_0909_5413_gb300 import rbf

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mode = args.mode or "mixed"
    probs = batch_problems(args)
    xy_np, f_np, ptr, params, rasm64 = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP64)
    _, _, _, _, rasm32 = rbf.batch_arrays(probs, factor_precision=rbf.RBF_FP32)
    ptr_c, params_c, rasm64_c = rbf.batch_ctypes(ptr, params, rasm64)
    rasm32_c = rbf.batch_ctypes(ptr, params, rasm32)[2]
    nprob, ntot = len(probs), ptr[-1]
    xy = torch.from_numpy(xy_np).cuda()
    f = torch.from_numpy(f_np).cuda()
    w = torch.zeros(ntot, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ctx = rbf.Context(local)
    h = ctx.handle
    if args.no_store:   # every FP64 product evaluates its pairs (nothing kept)
        rbf.rbf_set_option(h, rbf.RBF_OPT_STORE_F64, 0)

    def sparams(md):
        return rbf.RbfSolveParams(1e-13, 30, args.max_iters, int(md == "mixed"), args.max_iters, 1e-5,
                                  args.inner_cutoff if md == "mixed" else 0.0)

    def step(md, xy_t=xy, f_t=f, w_t=w):
        w_t.zero_()
        rbf.rbf_bin_batch(h, xy_t, ptr_c, params_c)
        rbf.rbf_rasm_setup_batch(h, rasm32_c if md == "mixed" else rasm64_c)
        return rbf.rbf_solve_batch(h, f_t, w_t, sparams(md), nprob, check=False)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, reps):
        ts, last = [], None
        for _ in range(reps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            last = fn()
            e1.record()
            barrier()
            ts.append(e0.elapsed_time(e1))
        return ts, last

    for _ in range(args.warmup):
        flush.zero_()
        step(mode)
    torch.cuda.synchronize()
    launches0 = ctx.launches
    clocks = ClockSampler(local)
    clocks.start()
    times, (st, infos) = timed(lambda: step(mode), args.steps)
    clk = clocks.stop()
    launches = ctx.launches - launches0
    ms = max_over_ranks(statistics.mean(times), dist, "cuda")
    summ = batch_summary(probs, infos)
    w_host = w.cpu().numpy()
    iters = [i.iters for i in infos]

    # FP64 matvec over the whole batch (every problem active), kernel time from the profiler
    rbf.rbf_profile_enable(h, True)
    for k in range(rbf.RBF_PROF_COUNT):
        rbf.rbf_profile_read(h, k)
    y = torch.empty_like(w)
    for _ in range(5):
        flush.zero_()
        rbf.rbf_matvec(h, w, y)
    torch.cuda.synchronize()
    n_mv, t_mv = rbf.rbf_profile_read(h, rbf.RBF_PROF_MATVEC_F64)
    rbf.rbf_profile_enable(h, False)
    pairs = rbf.rbf_count_neighbors(h)
    avg_s = t_mv / max(n_mv, 1) / 1e3
    roofline = f64_matvec_roofline(pairs, avg_s, n_mv, None, note="all problems of the batch in one launch")

    # the same batch with the Arnoldi step as separate kernels instead of the
    # fused persistent launch (the results must agree bit for bit)
    forms = None
    if not args.no_extra and mode == "mixed":
        forms = {}
        for name_, opt in (("separate_kernels", 0), ("fused_always", 1)):
            rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, opt)
            step(mode)
            ts, (st3, _) = timed(lambda: step(mode), 1)
            forms[name_] = {"ms_per_step": ts[0], "status": st3,
                            "bit_identical_to_timed": bool(np.array_equal(w.cpu().numpy(), w_host))}
        rbf.rbf_set_option(h, rbf.RBF_OPT_FUSED_STEP, 2)

    # the other precision, batched
    extra = None
    if not args.no_extra:
        other = "f64" if mode == "mixed" else "mixed"
        step(other)
        ts, (st2, inf2) = timed(lambda: step(other), max(1, min(args.steps, 2)))
        extra = {"precision": other, "ms_per_step": statistics.mean(ts), "status": st2,
                 **batch_summary(probs, inf2)}

    # the plain single-problem FP64 path, one problem at a time, on a seeded sample
    seq = None
    if not args.no_extra:
        sample = np.random.default_rng(7).choice(nprob, size=min(64, nprob), replace=False)
        sctx = rbf.Context(local)
        tot, sts = 0.0, []
        for k in sample:
            p = probs[k]
            cfg = rbf.config_for(p, max_iters=args.max_iters)
            xs = torch.from_numpy(p.xy).cuda()
            fs = torch.from_numpy(p.f).cuda()
            ws_ = torch.zeros(p.n, dtype=torch.float64, device="cuda")

            def one():
                sctx.bin(xs, cfg)
                sctx.rasm_setup(cfg)
                return sctx.solve(fs, ws_, cfg, check=False)
            ts, (s1, _) = timed(one, 1)
            tot += ts[0]
            sts.append(s1)
        sctx.close()
        ns = np.array([p.n for p in probs], dtype=np.float64)
        seq = {"precision": "f64", "sample_problems": len(sample), "sample_ms": tot,
               "projected_ms": tot * nprob / len(sample), "sample_converged": int(sum(1 for s in sts if s == 0)),
               "note": "single-problem solver (rbf_bin / rbf_rasm_setup / rbf_solve) per problem, "
                       "projected to the batch by problem count"}

    # end to end: pinned host inputs copied in, the three batch calls, w copied out
    e2e = None
    if not args.no_e2e:
        xy_h = torch.from_numpy(xy_np.copy()).pin_memory()
        f_h = torch.from_numpy(f_np.copy()).pin_memory()
        w_h = torch.zeros(ntot, dtype=torch.float64).pin_memory()
        xy_d, f_d, w_d = torch.empty_like(xy), torch.empty_like(f), torch.empty_like(w)

        def e2e_step():
            xy_d.copy_(xy_h, non_blocking=True)
            f_d.copy_(f_h, non_blocking=True)
            r = step(mode, xy_d, f_d, w_d)
            w_h.copy_(w_d, non_blocking=True)
            return r
        e2e_step()
        te, _ = timed(e2e_step, max(1, min(args.steps, 2)))
        e2e = {"value": statistics.mean(te), "unit": UNIT, "h2d_bytes_per_step": (xy_h.numel() + f_h.numel()) * 8,
               "d2h_bytes_per_step": w_h.numel() * 8}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_batch_sample(probs, budget_s=15.0, seed=0, w_gpu=w_host, ptr=ptr, iters=iters)

    if rank == 0:
        out = {"metric": BATCH_METRIC, "value": ms, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if mode == "f64" else "f32-inner/f64-outer", "data": "synthetic",
               "config": batch_config(args, probs, mode), "status": st, "solve": summ,
               "problems_per_s": nprob / (ms / 1e3), "points_per_s": ntot / (ms / 1e3),
               "step_ms": [round(t, 3) for t in times], "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clk, "other_precision": extra,
               "arnoldi_step": {"timed": "fused once at most 64 problems are active, separate kernels before",
                                "other_forms": forms},
               "one_problem_at_a_time": seq}
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ serving

SERVE_METRIC = "RBF serve latency p50 at 1e-13 rel. residual (Poisson arrivals, mixed precision)"


def serve_problems(args):
    return W.batch_workload(args.requests, lo=1000, hi=4_000_000, seed=W.DEFAULT_SEED + 5000)


def serve_config(args, probs) -> dict:
    ns = np.array([p.n for p in probs])
    return {"workload": "serve", "description": WORKLOADS["serve"][1], "requests": len(probs),
            "n_points_total": int(ns.sum()), "n_min": int(ns.min()), "n_max": int(ns.max()),
            "cutoff_sigmas": 8.6, "rasm": "4x4 lattice-point cores + 1-point ring (FP32 inverses)",
            "gmres_restart": 30, "rtol": 1e-13, "max_iters_per_request": args.max_iters,
            "precision": "mixed", "inner_cutoff_sigmas": args.inner_cutoff, "slots": args.slots, "rates": args.rates,
            "l2": "inputs (2.4-96 MB per request, 1.5 GB per sweep) far above L2", "parallelism": "replicas"}


def pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def run_reference_serve(args, ws, rank):
    if rank != 0:
        return
    probs = serve_problems(args)
    times, wall, cb = [], [], None
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = oracle_batch_sample(probs, budget_s=4.0, seed=step, max_n=300_000)
        if step >= args.warmup:
            times.append(cb["value"] / len(probs))
            wall.append((time.perf_counter() - t0) * 1e3)
    v = statistics.mean(times)
    cb["value"] = v
    cb["sample"] += "; value is the projected oracle time per request (one request at a time)"
    out = {"impl": "reference", "metric": SERVE_METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(wall),
           "ms_per_step_is": "wall time of one step's oracle sample (value is the per-request time it projects)",
           "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": serve_config(args, probs), "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def serve_sweep(rbf, args, local, probs, rates, warm: int) -> dict:
    """Serve the requests: warm-up (every slot grows its resident buffers on the
    largest request), a saturated burst (everything submitted at once), then
    Poisson arrivals at each fraction of the saturated rate."""
    R = len(probs)
    # pinned host buffers, as a serving front end would hold them
    import torch
    host = []
    for p in probs:
        xy = torch.from_numpy(p.xy.copy()).pin_memory().numpy()
        f = torch.from_numpy(p.f.copy()).pin_memory().numpy()
        w = torch.zeros(p.n, dtype=torch.float64).pin_memory().numpy()
        cfg = rbf.config_for(p, mixed=True, factor_precision=rbf.RBF_FP32, max_iters=args.max_iters,
                             max_refine=args.max_iters, inner_cutoff=args.inner_cutoff)
        host.append((xy, f, w, cfg))
    srv = rbf.Server(local, slots=args.slots)

    def submit(k):
        xy, f, w, cfg = host[k]
        return srv.submit(xy, f, cfg, w=w)

    def collect(tickets):
        out = {}
        for k, t in tickets.items():
            st, r, _ = srv.wait(t)
            out[k] = r
        return out

    big = int(np.argmax([p.n for p in probs]))
    for _ in range(max(1, warm)):
        collect({j: submit(big) for j in range(args.slots)})
    clocks = ClockSampler(local)
    clocks.start()
    s0 = srv.stats()
    t0 = srv.clock()
    res = collect({k: submit(k) for k in range(R)})
    t1 = max(r.t_done for r in res.values())
    sat = {"rate_per_s": None, "makespan_s": t1 - t0, "throughput_per_s": R / (t1 - t0),
           "p50_ms": pct([(r.t_done - r.t_submit) * 1e3 for r in res.values()], 50),
           "p99_ms": pct([(r.t_done - r.t_submit) * 1e3 for r in res.values()], 99)}
    thr = sat["throughput_per_s"]
    rows = []
    rng = np.random.default_rng(11)
    for frac in rates:
        lam = frac * thr
        gaps = rng.exponential(1.0 / lam, size=R)
        order = rng.permutation(R)
        tickets = {}
        start = srv.clock()
        at = start
        for k, g in zip(order, gaps):
            at += g
            while srv.clock() < at:
                time.sleep(min(0.002, max(0.0, at - srv.clock())))
            tickets[int(k)] = submit(int(k))
        rr = collect(tickets)
        lat = [(r.t_done - r.t_submit) * 1e3 for r in rr.values()]
        qd = [(r.t_admit - r.t_submit) * 1e3 for r in rr.values()]
        end = max(r.t_done for r in rr.values())
        rows.append({"rate_frac": frac, "rate_per_s": lam, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                     "mean_ms": float(np.mean(lat)), "queue_p50_ms": pct(qd, 50), "queue_p99_ms": pct(qd, 99),
                     "throughput_per_s": R / (end - start),
                     "converged": int(sum(1 for r in rr.values() if r.status == 0))})
    clk = clocks.stop()
    s1 = srv.stats()
    conv = [r for r in res.values() if r.status == 0]
    summ = {"converged": len(conv), "stagnated": int(sum(1 for r in res.values() if r.info.stagnated)),
            "not_converged": R - len(conv),
            "relres_max_converged": max((r.info.relres for r in conv), default=None),
            "iters_median": pct([r.info.iters for r in res.values()], 50),
            "peak_resident_gb": s1["peak_resident_bytes"] / 1e9, "mem_budget_gb": s1["mem_budget"] / 1e9,
            "trims": s1["trims"]}
    iters = [res[k].info.iters for k in range(R)]
    w_all = np.concatenate([host[k][2] for k in range(R)])
    srv.close()
    return {"saturated": sat, "rates": rows, "solve": summ, "iters": iters, "w_all": w_all, "clocks": clk,
            "launches": s1["launches"] - s0["launches"], "big": big}


def run_serve(args, ws, rank, local):
    import torch

    from paper_0909_5413_gb300 import rbf

    torch.cuda.set_device(local)
    probs = serve_problems(args)
    R = len(probs)
    res = serve_sweep(rbf, args, local, probs, [float(x) for x in args.rates.split(",") if x.strip()], args.warmup)
    rows, sat = res["rates"], res["saturated"]
    ptr = np.concatenate([[0], np.cumsum([p.n for p in probs])])

    # FP64 matvec roofline on the largest request (whole problem in one launch)
    roofline = matvec_roofline(rbf, probs[res["big"]], local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_batch_sample(probs, budget_s=15.0, seed=0, w_gpu=res["w_all"], ptr=ptr, iters=res["iters"],
                                  max_n=300_000)
        cpu["value"] /= R
        cpu["sample"] += "; value is the projected oracle time per request (one request at a time)"
    main = rows[0] if rows else sat
    h2d = float(np.mean([p.n * 24 for p in probs]))
    out = {"metric": SERVE_METRIC, "value": main["p50_ms"], "unit": UNIT, "n_gpus": ws, "steps": R,
           "warmup": args.warmup, "ms_per_step": main["mean_ms"] if rows else None, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32-inner/f64-outer", "data": "synthetic",
           "config": serve_config(args, probs), "p99_ms": main["p99_ms"], "rates": rows, "saturated": sat,
           "solve": res["solve"], "roofline": roofline, "cpu_baseline": cpu,
           "e2e": {"value": main["p50_ms"], "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d / 3,
                   "note": "the serving path is host to host: pinned inputs in, w out, per request"},
           "gpu_launches": res["launches"], "clocks": res["clocks"]}
    if rank == 0:
        print(json.dumps(out), flush=True)


def matvec_roofline(rbf, p, local) -> dict:
    import torch
    ctx = rbf.Context(local)
    cfg = rbf.config_for(p)
    ctx.bin(torch.from_numpy(p.xy).cuda(), cfg)
    w = torch.from_numpy(p.f).cuda()
    y = torch.empty_like(w)
    h = ctx.handle
    rbf.rbf_matvec(h, w, y)
    torch.cuda.synchronize()
    rbf.rbf_profile_enable(h, True)
    for _ in range(5):
        rbf.rbf_matvec(h, w, y)
    torch.cuda.synchronize()
    n_mv, t_mv = rbf.rbf_profile_read(h, rbf.RBF_PROF_MATVEC_F64)
    pairs = rbf.rbf_count_neighbors(h)
    ctx.close()
    avg_s = t_mv / max(n_mv, 1) / 1e3
    return f64_matvec_roofline(pairs, avg_s, n_mv, None, note=f"largest request, N={p.n}")


# ------------------------------------------------- paper-parameter variant

PAPER_METRIC = "RBF solve time at 1e-13 rel. residual, paper subdomain sizes (B = 5 sigma, D = 1.9 B)"


def run_paper(args, ws, rank, local):
    import torch

    from paper_0909_5413_gb300 import rbf

    torch.cuda.set_device(local)
    g = np.linspace(0.0, 1.0, 2048)
    gx, gy = np.meshgrid(g, g)
    xe_h = np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel()], axis=1))
    xe = torch.from_numpy(xe_h).cuda()
    exact = W.franke(xe_h[:, 0], xe_h[:, 1])
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    rows, times_all = [], []
    clocks = ClockSampler(local)
    clocks.start()
    launches = 0
    for ratio in (0.8, 0.9, 1.0):
        p = W.unit_square_problem(ratio, sigma=args.sigma, seed=W.DEFAULT_SEED)
        xy = torch.from_numpy(p.xy).cuda()
        f = torch.from_numpy(p.f).cuda()
        row = {"h_over_sigma": ratio, "n_points": p.n}
        for additive in (False, True):
            cfg = rbf.config_for(p, additive=additive)
            ctx = rbf.Context(local)
            w = torch.zeros(p.n, dtype=torch.float64, device="cuda")

            def step():
                w.zero_()
                ctx.bin(xy, cfg)
                ctx.rasm_setup(cfg)
                return ctx.solve(f, w, cfg, check=False)
            for _ in range(args.warmup):
                step()
            l0 = ctx.launches
            ts = []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st, info = step()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            key = "asm" if additive else "rasm"
            row[key] = {"ms": statistics.mean(ts), "iters": info.iters, "relres": info.relres, "status": st}
            launches += ctx.launches - l0
            if not additive:
                times_all.append(statistics.mean(ts))
                s = torch.empty(xe_h.shape[0], dtype=torch.float64, device="cuda")
                rbf.rbf_eval(ctx.handle, xe, xe_h.shape[0], w, s)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                rbf.rbf_eval(ctx.handle, xe, xe_h.shape[0], w, s)
                e1.record()
                torch.cuda.synchronize()
                err = np.abs(s.cpu().numpy() - exact)
                row["eval"] = {"points": int(xe_h.shape[0]), "ms": e0.elapsed_time(e1),
                               "max_abs_error_vs_franke": float(err.max()),
                               "rms_error_vs_franke": float(np.sqrt(np.mean(err ** 2)))}
            ctx.close()
        rows.append(row)
    clk = clocks.stop()
    if rank == 0:
        v = times_all[1]   # h/sigma = 0.9, the paper's main case
        out = {"metric": PAPER_METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "paper", "description": WORKLOADS["paper"][1], "sigma": args.sigma,
                          "value_is": "RASM solve (bin + setup + GMRES) at h/sigma = 0.9",
                          "l2": "flushed (256 MB write) before each timed step", "parallelism": "replicas"},
               "rows": rows, "roofline": None, "cpu_baseline": None,
               "e2e": None, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    kind = "batch" if args.workload.startswith("batch") else (args.workload if args.workload in ("serve", "paper")
                                                                else "one")
    if args.impl == "reference":
        if kind == "paper":
            print(json.dumps({"impl": "reference", "unavailable": "the paper workload is reported by the GPU arm only; "
                              "its oracle comparison is in the tests"}), flush=True)
            return
        {"batch": run_reference_batch, "serve": run_reference_serve, "one": run_reference}[kind](args, ws, rank)
        return
    {"batch": run_batch, "serve": run_serve, "paper": run_paper, "one": run_ours}[kind](args, ws, rank, local)


if __name__ == "__main__":
    main()
