"""Multi-GPU is replicas only: every rank renders its own copy of the workload and
the job's rate is all ranks' rays over the slowest rank's step time.  The
reduction bench.py applies is checked here with two gloo ranks on the CPU
(127.0.0.1 rendezvous), each reporting a different step time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.reduce_step_time(times[rank], "cpu")
        rays = 1000 * world / (ms * 1e-3) / 1e6
        out[rank] = (ms, rays)
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    world, times = 2, [3.0, 4.5]
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == max(times)
        assert rate == pytest.approx(1000 * world / (max(times) * 1e-3) / 1e6)


def test_single_process_keeps_its_time():
    import bench
    assert bench.reduce_step_time(2.5, "cpu") == 2.5
