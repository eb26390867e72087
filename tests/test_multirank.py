"""The benchmark's multi-rank path, on CPU with gloo (world size 2).

One generator per rank (replicas: a single pool does not shard, since every
pass gathers across the whole pool); ranks get different streams through the
stream id appended to the seed (Section 8's processor number); the job's
time is the slowest rank's and its units are the sum over ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    from oracle import py_oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank
    units_local = 1000 * (rank + 1)
    ms, units = bench.reduce_over_ranks(ms_local, units_local, dist, "cpu")
    # each rank's replica: same seed, stream id = rank
    g = orc.Generator(4, 256, 7, 0.5, stream=rank)
    head = g.fill(64)
    gathered = [torch.zeros(64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(head.astype(np.float32)))
    q.put((rank, ms, units, [t.numpy().copy() for t in gathered]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_and_distinct_streams():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, heads in res:
        assert ms == 15.0            # slowest rank
        assert units == 3000         # all ranks' work
        assert not np.array_equal(heads[0], heads[1])   # different streams per rank


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 42, None, "cpu") == (3.5, 42)
