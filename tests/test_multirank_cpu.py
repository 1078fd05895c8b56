"""The N > 1 bench path on CPU: two gloo ranks, each timing its own
independent signal; the job's time is the slowest rank's and its units the
sum over ranks (weak scaling, no data-path collective)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank            # per-rank timed-region length
    det = 1000.0 + rank                 # per-rank detected coefficients
    q.put((rank, bench.reduce_scalar(ms, "max", world), bench.reduce_scalar(det, "sum", world),
           bench._dist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, (w, r, local) in out:
        assert mx == 150.0 and sm == 2001.0
        assert (w, r, local) == (2, rank, rank)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_scalar(3.5, "max", 1) == 3.5
    assert bench.reduce_scalar(7.0, "sum", 1) == 7.0
