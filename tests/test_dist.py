"""The N>1 bench path on CPU: world_size-2 gloo ranks run the barrier,
max-over-ranks and sum that bench.py uses under torchrun (pairs are
independent, so the data path has no collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    mx = d.max(10.0 * (rank + 1))          # per-rank step time: the job takes the slowest
    total = d.sum(1000.0 * (rank + 1))     # cells: the job counts every rank's pairs
    d.barrier()
    d.close()
    q.put((rank, mx, total, bench.dist_env()))


def test_two_rank_max_and_sum():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, total, env in got:
        assert mx == 20.0
        assert total == 3000.0
        assert env == (world, rank, rank)


def test_single_process_dist_is_a_no_op():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    d = bench.Dist("gloo")
    assert not d.on
    assert d.max(3.5) == 3.5 and d.sum(2.0) == 2.0
    d.barrier()
