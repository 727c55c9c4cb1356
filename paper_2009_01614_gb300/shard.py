"""Row-sharded exact k-NN over several processes (one per GPU).

The collection is split into contiguous row ranges; every rank answers the
query exactly on its own range, the k (distance, row) pairs of all ranks are
all-gathered (one collective of 12 k bytes per query and rank), and each rank
merges them by (distance, row).  Rows are global: local row + the shard's first
row.  The exact answer of the whole collection is the merge of the shards'
exact answers, because every row of the global top-k is in its own shard's
top-k.  Cross-shard ties are ordered by the returned (fp32) distance, then by
row.
"""
import numpy as np


def shard_range(N, rank, world):
    """Rows [r0, r1) of shard `rank` of `world` over N rows."""
    return N * rank // world, N * (rank + 1) // world


def merge_knn(idx_parts, dist_parts, k):
    """Merge per-shard answers (lists of [B, k_i] global rows and distances)
    into the k smallest by (distance, row): ([B, k] int64, [B, k] float32)."""
    idx = np.concatenate([np.asarray(p, dtype=np.int64) for p in idx_parts], axis=1)
    dist = np.concatenate([np.asarray(p, dtype=np.float32) for p in dist_parts], axis=1)
    B = idx.shape[0]
    out_i = np.empty((B, k), np.int64)
    out_d = np.empty((B, k), np.float32)
    for b in range(B):
        valid = idx[b] >= 0
        order = np.lexsort((idx[b][valid], dist[b][valid]))[:k]
        out_i[b] = idx[b][valid][order]
        out_d[b] = dist[b][valid][order]
    return out_i, out_d


def sharded_knn(local_search, Q, k, N, rank, world, group=None):
    """Exact k-NN of queries Q [B, n] over a collection sharded across the
    ranks of torch.distributed (`group`): local_search(Q, k) returns this
    rank's (local rows [B, k'], distances [B, k']) with k' = min(k, shard
    rows); every rank returns the merged global answer."""
    import torch
    import torch.distributed as dist
    r0, r1 = shard_range(N, rank, world)
    kk = min(k, r1 - r0)
    li, ld = local_search(Q, kk)
    B = len(Q)
    gi = np.full((B, k), -1, np.int64)
    gd = np.full((B, k), np.inf, np.float32)
    gi[:, :kk] = np.asarray(li, dtype=np.int64) + r0
    gd[:, :kk] = np.asarray(ld, dtype=np.float32)
    ti, td = torch.from_numpy(gi), torch.from_numpy(gd)
    all_i = [torch.empty_like(ti) for _ in range(world)]
    all_d = [torch.empty_like(td) for _ in range(world)]
    dist.all_gather(all_i, ti, group=group)
    dist.all_gather(all_d, td, group=group)
    return merge_knn([t.numpy() for t in all_i], [t.numpy() for t in all_d], k)
