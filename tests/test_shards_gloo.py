"""Multi-rank host logic on CPU: two gloo ranks (no GPU).

Row shards answered independently and concatenated in rank order equal the answer
over the whole table (Sec. 3.1); the slowest rank's time is what counts. The local
scan here is the CPU oracle, standing in for each rank's GPU scan.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_1801_03644_gb300 import shards
    from paper_1801_03644_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.mixed_clustered(n=40_001, nq=12)
        lo, hi = shards.row_range(wl.n, rank, world)
        res = []
        for query in wl.queries:
            local = oracle.mdrq([c[lo:hi] for c in wl.columns], query, 2)
            res.append(shards.gather_shard_answer(local, lo))
        slowest = shards.max_over_ranks(1.5 + rank)
        q.put((rank, [r.tolist() for r in res], slowest))
    finally:
        dist.destroy_process_group()


def test_row_shards_concatenate_to_the_whole_answer():
    import oracle
    from paper_1801_03644_gb300 import workloads as W
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = W.mixed_clustered(n=40_001, nq=12)
    want = [oracle.mdrq(wl.columns, query, 2).tolist() for query in wl.queries]
    for rank, res, slowest in got:
        assert res == want
        assert slowest == 2.5


def test_row_range_covers_rows_once():
    from paper_1801_03644_gb300 import shards
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            rr = [shards.row_range(n, r, world) for r in range(world)]
            assert rr[0][0] == 0 and rr[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
            assert max(h - l for l, h in rr) - min(h - l for l, h in rr) <= 1
