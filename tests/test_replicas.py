"""The multi-GPU bench path is replicas only: every rank builds and evaluates its own copy
of the workload with no collective on the data path; the job's step time is the largest
over the ranks and its value counts every replica. Checked with two gloo ranks on the CPU
(the reduction the bench runs over NCCL on GPUs)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step, ev = bench.job_times([10.0 + 5.0 * rank, 8.0 - rank], dist, "cpu")
    out[rank] = (step, ev, bench.job_value(1000, 48, world, step))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        step, ev, value = out[r]
        assert step == 15.0 and ev == 8.0  # the slowest rank's times, on every rank
        assert value == pytest.approx(1000 * 48 * 2 / 15e-3)


def test_single_process_passes_through_and_reference_arm_runs_on_rank0_only(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_times([3.0, 4.0]) == [3.0, 4.0]
    monkeypatch.setenv("RANK", "1")
    # ranks other than 0 leave the reference arm at once, without work or output
    assert bench.run_reference(None) is None
