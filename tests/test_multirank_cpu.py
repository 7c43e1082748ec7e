"""The multi-rank path of bench.py on CPU: two gloo ranks combine their
timings and counts as the benchmark does on N GPUs (the slowest rank's time,
the sum of the ranks' converged pairs), with no other collective."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, pairs = bench.combine_ranks(100.0 + 25.0 * rank, 200 * (rank + 1), dist, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{ms} {pairs}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, pairs = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert ms == 125.0          # max over ranks
        assert pairs == 600.0       # 200 + 400


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.combine_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)
