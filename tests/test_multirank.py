"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1
agree on the job's time (the slowest rank's) and on the job's throughput
(every rank searches its own replica, so the queries add up)."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [40.0, 55.0][rank]
        job_ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
        dist.barrier()
        value = bench.job_throughput(1000, 3, world, job_ms)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{job_ms} {value}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_throughput(tmp_path):
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(2)]
    assert got[0] == got[1]
    job_ms, value = got[0]
    assert job_ms == 55.0
    assert value == pytest.approx(2 * 1000 * 3 / 0.055)


def test_one_rank_is_its_own_job():
    import torch

    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
    assert bench.job_throughput(10_000, 20, 1, 61.7) == pytest.approx(10_000 * 20 / 0.0617)
