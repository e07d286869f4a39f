"""The multi-process (replica) path of bench.py on CPU: two gloo ranks agree on the job's
step time (the slowest rank) and its work (the sum), exactly as the NCCL ranks do."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, blends = bench.job_totals(ms_step=2.0 + rank, blends=1000 * (rank + 1), world=world, device="cpu")
    out[rank] = (ms, blends)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_report_max_time_and_total_work():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (3.0, 3000.0)


def test_single_process_is_the_identity():
    import bench
    assert bench.job_totals(1.5, 42, 1, "cpu") == (1.5, 42.0)
