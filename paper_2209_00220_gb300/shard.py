"""Row-range shards of one column over several ranks (one GPU per rank).

Rows are independent under a scan and a lookup, so a column splits into
contiguous row ranges, one per rank, each a whole number of 1024-row tiles:
every shard's result bit vector is then a whole number of 32-bit words and the
shards' bit vectors concatenate to the whole column's. For the shards to agree
on codes, the dictionary and the PP-VBS codes (Algorithm 1) are built from the
whole column's values and counts -- gathered from the ranks -- and every shard
is encoded against them (`domain_values` + `domain_counts`). The only exchange
on the query path is one 64-bit selected-row count per rank, whose exclusive
prefix places each rank's lookup output in the whole column's output order.
"""
from __future__ import annotations

import numpy as np

TILE_ROWS = 1024


def shard_range(n: int, world: int, rank: int, align: int = TILE_ROWS) -> tuple[int, int]:
    """Rows [lo, hi) of `rank`: tiles dealt out in contiguous blocks as evenly
    as the tile count allows (a rank may get none)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    tiles = (n + align - 1) // align
    base, extra = divmod(tiles, world)
    t0 = rank * base + min(rank, extra)
    t1 = t0 + base + (1 if rank < extra else 0)
    return min(n, t0 * align), min(n, t1 * align)


def local_dictionary(values) -> tuple[np.ndarray, np.ndarray]:
    """Sorted distinct values of this shard and their counts."""
    a, q = np.unique(np.asarray(values, dtype=np.int32), return_counts=True)
    return a.astype(np.int32), q.astype(np.uint64)


def merge_dictionaries(parts) -> tuple[np.ndarray, np.ndarray]:
    """Union of (values, counts) pairs, counts of equal values summed."""
    parts = [p for p in parts if len(p[0])]
    if not parts:
        return np.zeros(0, np.int32), np.zeros(0, np.uint64)
    a = np.concatenate([np.asarray(p[0], dtype=np.int32) for p in parts])
    q = np.concatenate([np.asarray(p[1], dtype=np.uint64) for p in parts])
    u, inv = np.unique(a, return_inverse=True)
    tot = np.zeros(u.size, np.uint64)
    np.add.at(tot, inv, q)
    return u.astype(np.int32), tot


def _dist(group):
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return None
    return dist


def global_dictionary(shard_values, group=None) -> tuple[np.ndarray, np.ndarray]:
    """The whole column's dictionary and counts, from every rank's shard (an
    all-gather of the per-shard dictionaries; the shard's own when not
    distributed)."""
    mine = local_dictionary(shard_values)
    dist = _dist(group)
    if dist is None or dist.get_world_size(group) == 1:
        return mine
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, (mine[0].tolist(), mine[1].tolist()), group=group)
    return merge_dictionaries([(np.array(p[0], np.int32), np.array(p[1], np.uint64)) for p in parts])


def encode_shard(B, shard_values, layout: str, dictionary, **opts):
    """Encodes a shard against the whole column's dictionary (values, counts):
    PP-VBS codes from the whole column's counts, ByteSlice / Bit-Packed codes
    = rank in the whole column's dictionary (unless the caller declares
    domain_bits, which needs no dictionary)."""
    a, q = dictionary
    if layout == "ppvbs":
        return B.bs_encode_column(shard_values, layout, domain_values=a, domain_counts=q, **opts)
    if opts.get("domain_bits"):
        return B.bs_encode_column(shard_values, layout, **opts)
    return B.bs_encode_column(shard_values, layout, domain_values=a, **opts)


def output_offset(count: int, group=None) -> tuple[int, int]:
    """(exclusive prefix of the ranks' selected-row counts at this rank, total)."""
    dist = _dist(group)
    if dist is None or dist.get_world_size(group) == 1:
        return 0, int(count)
    counts = [None] * dist.get_world_size(group)
    dist.all_gather_object(counts, int(count), group=group)
    r = dist.get_rank(group)
    return int(sum(counts[:r])), int(sum(counts))
