"""The multi-rank path of bench.py on CPU: two gloo ranks split independent LTs
without any collective on the data path, and the timing reduction takes the
maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist()
    mine = list(bench.shard(10, world, rank))
    got = d.max(float(rank + 1) * 1.5)
    d.barrier()
    q.put((rank, mine, got))
    d.close()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == [0, 1, 2, 3, 4] and res[1][1] == [5, 6, 7, 8, 9]
    assert res[0][2] == res[1][2] == 3.0


def test_shard_covers_everything_once():
    import bench
    for total in [0, 1, 7, 64, 129]:
        for world in [1, 2, 3, 8]:
            seen = [u for r in range(world) for u in bench.shard(total, world, r)]
            assert seen == list(range(total))
