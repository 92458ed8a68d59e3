"""The multi-GPU path of bench.py is replicas (one independent solve per rank, no data
exchanged): its host logic -- a barrier, then the job's time as the maximum over ranks and the
units summed over ranks -- runs here as two gloo processes on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r took 1 + r seconds for 100 units (the slowest rank sets the job's time)
        total_s, rate = bench.replica_rate(1.0 + rank, 100.0, world, device="cpu")
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{total_s} {rate}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_summed_units(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        total_s, rate = (float(x) for x in open(tmp_path / f"rank{rank}.txt").read().split())
        assert total_s == 2.0          # max over ranks of 1.0 and 2.0
        assert rate == 2 * 100.0 / 2.0  # units of both ranks over the job's time


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(0.5, 10.0, 1) == (0.5, 20.0)
