"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
frame shard; the timer reduction takes the max over ranks and the work the
sum (no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    red = bench.RankReduce(dist, "cpu")
    red.barrier()
    seed = bench.rank_seed(1, rank)
    wl = synth.make_workload("rm26_crc6", 1.0, 64, seed=seed)
    mx = red.max(10.0 + rank)
    sm = red.sum(100 * (rank + 1))
    q.put((rank, seed, wl.y[:2].tolist(), mx, sm))
    dist.destroy_process_group()


def test_two_rank_reduction_and_disjoint_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [1, 2]
    assert not np.array_equal(np.array(res[0][2]), np.array(res[1][2]))
    assert all(r[3] == 11.0 for r in res)
    assert all(r[4] == 300.0 for r in res)
