"""The multi-GPU form of the benchmark is "replicas only": every rank runs its own copy of
the workload, and the reported value is the total work over the slowest rank's time.  The
host-side logic of that (barrier, max over ranks) runs here as world-size-2 gloo ranks on
the CPU; no GPU and no data-path collective are involved."""
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


def _rank_main(rank, world, port, elapsed, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        slowest = bench.max_over_ranks(world, elapsed[rank])
        out[rank] = slowest
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    elapsed = [1.25, 3.5]
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, elapsed, out), nprocs=world,
                           start_method="spawn", join=True)
        got = dict(out)
    # every rank sees the slowest rank's time, so value = world * units / slowest
    assert got == {0: 3.5, 1: 3.5}


def test_single_rank_needs_no_process_group():
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(1, 2.0) == 2.0
