"""Host logic for running the scan on several GPUs, one process per GPU.

Two ways to spread the work (torch.distributed, one rank per GPU):

* Query replicas (what ``bench.py --gpus N`` does): every rank holds the whole table
  and answers its own batch of queries; no data crosses ranks. Throughput adds up
  (weak scaling); ``max_over_ranks`` gives the slowest rank's time.
* Row shards (the horizontal partitioning of Sec. 3.1 with contiguous ranges): rank r
  holds rows ``row_range(n, r, world)`` and answers every query on its shard; the
  partial answers, shifted by the shard's first row, are concatenated in rank order
  (Sec. 3.1), which keeps the list ascending. ``gather_shard_answer`` is that
  exchange: an all-gather of the counts, then of the ids.
"""
from __future__ import annotations

import numpy as np


def row_range(n: int, rank: int, world: int) -> tuple:
    """Contiguous rows [lo, hi) of shard ``rank`` out of ``world``; sizes differ by <= 1."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside world %d" % (rank, world))
    return n * rank // world, n * (rank + 1) // world


def max_over_ranks(value: float, group=None) -> float:
    """The largest ``value`` over all ranks (the timing rule: the slowest rank counts)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_shard_answer(local_ids: np.ndarray, row_offset: int, group=None) -> np.ndarray:
    """Concatenate the ranks' shard answers in rank order (Sec. 3.1).

    ``local_ids``: this rank's ascending uint32 ids, relative to its shard;
    ``row_offset``: the shard's first row. Every rank receives the whole ascending
    answer. Exchange: all-gather of the counts, then an all-gather of the ids padded
    to the largest count.
    """
    import torch
    import torch.distributed as dist
    ids = np.asarray(local_ids, dtype=np.int64) + int(row_offset)
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return ids.astype(np.uint32)
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    cnt = torch.tensor([ids.size], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(1, max(counts))
    buf = torch.full((width,), -1, dtype=torch.int64, device=dev)
    if ids.size:
        buf[: ids.size] = torch.from_numpy(ids).to(dev)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = [p[:c].cpu().numpy() for p, c in zip(parts, counts)]
    return np.concatenate(out).astype(np.uint32) if out else np.zeros(0, np.uint32)
