"""The N > 1 path of bench.py on the CPU: two processes joined by a `gloo` process group.

bench.py under torchrun runs replicas: each rank solves its own seeded replica of the workload
with no data-path collective, and the job's time is the maximum over the ranks of their timed
regions.  These tests check that host logic without a GPU: the max-over-ranks reduction
(`bench.reduce_max`), the per-rank replica seeds, and that the reference arm runs on rank 0 only
(the other ranks return without work).
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        local = 10.0 + 7.5 * rank                    # this rank's timed region, ms
        job = bench.reduce_max(local, "cpu")
        # replica seeds: each rank's workload is its own seeded domain
        prob = bench.WORKLOADS["star2d_p2_n512"](rank)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
            fh.write(f"{job} {prob.shape.phase!r} {prob.shape.center!r}\n")
        if rank != 0:                                # the reference arm does nothing off rank 0
            class A:
                workload, steps, warmup = "disk2d_p1_n32", 1, 0
            assert bench.run_reference(A) is None
            with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as fh:
                fh.write("none\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_replicas(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    lines = [open(tmp_path / f"rank{r}.txt").read().split(" ", 1) for r in range(world)]
    jobs = [float(l[0]) for l in lines]
    assert jobs == [17.5, 17.5]                      # both ranks see the slowest rank's time
    assert lines[0][1] != lines[1][1]                # different seeded replicas
    assert open(tmp_path / "ref1.txt").read().strip() == "none"


def test_reduce_max_without_process_group():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_max(3.25, "cpu") == 3.25
