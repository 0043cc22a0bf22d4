"""Host logic of `bench.py --gpus N` (N independent replicas, no data-path
collective): every rank reports its own time, rank 0 takes the maximum, and the
throughput counts the units of all ranks.  Runs as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = 10.0 * (rank + 1)  # each replica's own elapsed time
    tmax = bench.max_over_ranks(t, world)
    out[rank] = tmax
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == 20.0 and out[1] == 20.0


def test_reference_arm_other_ranks_do_no_work():
    import bench

    class Args:
        steps, warmup, gpus, nx = 1, 0, 2, 64

    assert bench.run_reference(Args, 2, 1) == 0  # rank 1 exits without work
