"""Multi-process (N > 1) path of the benchmark on CPU: independent replicas
joined only by the max-over-ranks timing reduction (gloo, world size 2).
The solve itself has no data-parallel exchange on one box (replicas only)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 7.0 * rank          # each replica's timed total
        mx = bench.replica_max(local_ms, world, device="cpu")
        out[rank] = (mx, bench.replicas_value(world, 4096 * 16384, 10, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 17.0
    assert res[0][1] == pytest.approx(2 * 4096 * 16384 * 10 / 17.0e-3)


def test_single_replica_needs_no_collective():
    import bench
    assert bench.replica_max(12.5, 1) == 12.5
    assert bench.replicas_value(1, 100, 4, 2.0) == pytest.approx(100 * 4 / 2e-3)
