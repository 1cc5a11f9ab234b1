"""The N>1 paths on CPU: world_size-2 gloo ranks run the barrier,
max-over-ranks and sum that bench.py uses under torchrun (pairs are
independent, so the data path has no collective), and split one batch with
bsw_partition, each rank extending its part (with the oracle, standing in
for a device), the parts' results concatenated being the whole batch's."""
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


def _partition_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as td
    import numpy as np
    import oracle
    from paper_1907_12931_gb300 import bsw, workload as W
    td.init_process_group("gloo")
    wl = W.make("long10k", n_pairs=600)
    b = bsw.bsw_partition(wl.params, wl.q_len, wl.t_len, world)
    part = wl.subset(np.arange(b[rank], b[rank + 1]))
    res, cells, _ = oracle.extend_batch(part, nthreads=2)
    got = [None] * world
    td.all_gather_object(got, (rank, res, int(cells.sum())))
    td.barrier()
    td.destroy_process_group()
    if rank == 0:
        whole, wcells, _ = oracle.extend_batch(wl, nthreads=2)
        parts = [g[1] for g in sorted(got, key=lambda x: x[0])]
        q.put((bool(np.array_equal(np.concatenate(parts), whole)), [g[2] for g in got], int(wcells.sum()),
               b.tolist()))
    else:
        q.put(None)


def test_two_rank_partition_equals_whole():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_partition_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    equal, cells, whole_cells, bounds = [o for o in out if o is not None][0]
    assert equal
    assert sum(cells) == whole_cells
    assert bounds[0] == 0 and bounds[-1] == 600 and 0 < bounds[1] < 600
