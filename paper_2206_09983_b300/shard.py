"""Seed sharding across GPUs: the host-side gather of the shards' results.

Every rank holds one graph on its own GPU with ``Graph.set_shard(rank,
world)`` and inserts the same batches (each shard ingests the whole stream, so
every search sees the whole window).  A shard enumerates only the seeds it
owns, so its counts and lists are a disjoint part of the batch's result; the
job's result is the sum of the counts and the union of the lists.  The only
exchange is this gather on the host over a torch.distributed group (gloo, or
any group that can move Python objects): no device memory crosses GPUs.
"""
from __future__ import annotations

import numpy as np


def merge_counts(per_shard: list) -> list:
    """Per-query counts of the whole batch: the shards' counts summed."""
    if not per_shard:
        return []
    return [int(sum(c[q] for c in per_shard)) for q in range(len(per_shard[0]))]


def merge_rows(per_shard: list) -> np.ndarray:
    """The whole batch's rows of one (query, sign): the shards' rows (uint64
    rows of vertex ids then edge seqs) concatenated and sorted."""
    parts = [r for r in per_shard if len(r)]
    if not parts:
        return per_shard[0] if per_shard else np.empty((0, 0), dtype=np.uint64)
    rows = np.concatenate(parts, axis=0)
    return rows[np.lexsort(rows.T[::-1])]


def gather_batch(counts_pos: list, counts_neg: list, rows: dict | None = None, group=None,
                 dst: int = 0):
    """Gather one batch's shard results to rank `dst`.

    counts_pos / counts_neg: this shard's per-query counts; rows (optional):
    {(query, sign): uint64 rows} of this shard.  Returns, on `dst`, the merged
    (counts_pos, counts_neg, rows) of the whole batch; None elsewhere."""
    import torch.distributed as dist

    mine = (list(counts_pos), list(counts_neg), rows or {})
    world = dist.get_world_size(group)
    got = [None] * world if dist.get_rank(group) == dst else None
    dist.gather_object(mine, got, dst=dst, group=group)
    if got is None:
        return None
    keys = sorted({k for _, _, r in got for k in r})
    merged_rows = {k: merge_rows([r[k] for _, _, r in got if k in r]) for k in keys}
    return (merge_counts([g[0] for g in got]), merge_counts([g[1] for g in got]), merged_rows)
