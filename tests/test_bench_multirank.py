"""The multi-rank path of bench.py on CPU: gloo ranks, each with its own batch
of one seeded frame stream (batch b on rank b mod N); the timer reduction
takes the max over ranks and the work the sum (no data-path collective)."""
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
    first = bench.rank_first_frame(B, world, rank)
    wl = synth.make_workload("rm26_crc6", 1.0, B, seed=1, first_frame=first)
    mx = red.max(10.0 + rank)
    sm = red.sum(100 * (rank + 1))
    q.put((rank, first, wl.y.tolist(), mx, sm))
    dist.destroy_process_group()


B = 48  # frames per rank and step


@pytest.mark.parametrize("world", [2, 3])
def test_rank_reduction_and_round_robin_batches(world):
    import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # batch b of the stream on rank b mod world: disjoint frame ranges that tile [0, world B)
    assert [r[1] for r in res] == [B * r for r in range(world)]
    stream = synth.make_workload("rm26_crc6", 1.0, world * B, seed=1)
    assert np.array_equal(np.concatenate([np.array(r[2], np.float32) for r in res]), stream.y)
    # rank 0 decodes the frames a one-rank run decodes
    assert np.array_equal(np.array(res[0][2], np.float32), synth.make_workload("rm26_crc6", 1.0, B, seed=1).y)
    assert all(r[3] == 10.0 + world - 1 for r in res)
    assert all(r[4] == 100 * world * (world + 1) // 2 for r in res)


def test_shard_batches_partitions():
    import synth

    for total in (1, 5, 12):
        for world in (1, 2, 3, 8):
            parts = [synth.shard_batches(total, world, r) for r in range(world)]
            flat = sorted(b for p in parts for b in p)
            assert flat == list(range(total))
            assert all(b % world == r for r, p in enumerate(parts) for b in p)
