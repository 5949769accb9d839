"""The benchmark's multi-rank timing: every rank reports the slowest rank's
time (two gloo ranks on CPU; with one rank the value passes through)."""
import os
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"file://{os.path.join(out, 'init')}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.25 + 3.0 * rank, world, "cpu")
        with open(os.path.join(out, f"r{rank}"), "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    mp.start_processes(_worker, args=(2, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert float((tmp_path / f"r{r}").read_text()) == 4.25


def test_max_over_ranks_one_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
