"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): replicas only,
so the one collective is the max over ranks of the step time, and the
reference arm runs on rank 0 alone (the other ranks return without work)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_init(None)   # from the environment torchrun sets
        mine = 10.0 * (rank + 1) + 0.25
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        # the reference arm: ranks other than 0 return at once, before any work
        ran = "skipped"
        if rank != 0:
            ran = [bench.run_reference(None, ws, rank), bench.run_reference_batch(None, ws, rank),
                   bench.run_reference_serve(None, ws, rank)]
            ran = "None" if all(r is None for r in ran) else "work"
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
            fh.write(f"{got_ws} {got_rank} {got_local} {slowest} {ran}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_replicas_take_the_max_over_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(rank_main, args=(ws, free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(ws)]
    for r, row in enumerate(rows):
        assert row[:3] == [str(ws), str(r), str(r)]
        assert float(row[3]) == 20.25          # the slower replica's time, on every rank
    assert rows[1][4] == "None"                # rank 1 of the reference arm did nothing


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
