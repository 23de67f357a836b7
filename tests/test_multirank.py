"""The benchmark's multi-replica host logic on two CPU ranks (gloo): every
rank reports the slowest replica's time, and the job's throughput counts all
replicas' units over that time (replicas only: no collective touches the
data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        assert (r, w) == (rank, world)
        slowest = bench.max_over_ranks(times[rank], world, device="cpu")
        out[rank] = (slowest, bench.job_value(1000.0, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_replica():
    import torch.multiprocessing as mp
    world, times = 2, [0.004, 0.0055]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, value = res[rank]
        assert slowest == max(times)
        assert value == pytest.approx(1000.0 * world / max(times))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.01, 1) == 0.01
    assert bench.job_value(500.0, 1, 0.5) == 1000.0
