"""Multi-process path of bench.py on CPU: two gloo ranks, each solving its own
replica (no data-path collective); the reported time is the slowest rank's."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1304_5583_gb300 import synth
    try:
        local = 10.0 * (rank + 1)
        slowest = bench.max_over_ranks(local, world)
        w = synth.workload("tiny_20x30", seed=bench.replica_seed(0, rank))
        np.save(os.path.join(out, f"rank{rank}.npy"), np.concatenate([[slowest], w.M.ravel()]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_and_solve_distinct_replicas(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 20.0
    assert not np.array_equal(r0[1:], r1[1:])


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_seed(7, 0) == 7
