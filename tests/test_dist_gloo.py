"""Multi-rank host logic on CPU: two gloo ranks shard a scan's slices and reduce timings."""
import os
import socket

import pytest

from paper_1809_04195_gb300.dist import slice_shard

torch = pytest.importorskip("torch")


def test_slice_shard_covers_every_slice_once():
    for S in (0, 1, 7, 288, 320):
        for W in (1, 2, 3, 4, 8, 11):
            seen = []
            for r in range(W):
                a, n = slice_shard(S, r, W)
                seen.extend(range(a, a + n))
            assert seen == list(range(S))
            counts = [slice_shard(S, r, W)[1] for r in range(W)]
            assert max(counts) - min(counts) <= (1 if S else 0)
    with pytest.raises(ValueError):
        slice_shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1809_04195_gb300.dist import max_over_ranks, slice_shard, sum_over_ranks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, n = slice_shard(320, rank, world)
    wall = 1.5 + rank  # pretend rank r took 1.5 + r seconds
    q.put((rank, start, n, max_over_ranks(wall), sum_over_ranks(n)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r[1], r[2]) for r in res] == [(0, 160), (160, 160)]
    assert all(r[3] == 2.5 for r in res)  # slowest rank
    assert all(r[4] == 320 for r in res)  # every slice once
