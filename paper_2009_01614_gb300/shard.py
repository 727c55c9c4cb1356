"""Row-sharded exact k-NN over several processes (one per GPU).

The collection is split into contiguous row ranges; every rank answers the
query exactly on its own range and attaches, to each of its k answers, the
FP64 squared distance summed in the definition's order (isax_exact_d2 on the
GPU), the value the brute-force definition orders by.  The k (row, fp32
distance, FP64 squared distance) triples of all ranks are all-gathered (one
collective of 20 k bytes per query and rank) and each rank merges them by
(FP64 squared distance, global row).  Rows are global: local row + the shard's
first row.  The merge is the whole collection's exact answer: every row of the
global top-k is in its own shard's top-k, and the order is the definition's
order even where two rows of different shards have the same fp32 distance.
"""
import numpy as np


def shard_range(N, rank, world):
    """Rows [r0, r1) of shard `rank` of `world` over N rows."""
    return N * rank // world, N * (rank + 1) // world


def merge_knn(idx_parts, dist_parts, d2_parts, k):
    """Merge per-shard answers (lists of [B, k_i] global rows, fp32 distances
    and FP64 squared distances; rows < 0 are padding) into the k smallest by
    (FP64 squared distance, row): ([B, k] int64, [B, k] float32, [B, k] float64)."""
    idx = np.concatenate([np.asarray(p, dtype=np.int64) for p in idx_parts], axis=1)
    dist = np.concatenate([np.asarray(p, dtype=np.float32) for p in dist_parts], axis=1)
    d2 = np.concatenate([np.asarray(p, dtype=np.float64) for p in d2_parts], axis=1)
    B = idx.shape[0]
    out_i = np.empty((B, k), np.int64)
    out_d = np.empty((B, k), np.float32)
    out_d2 = np.empty((B, k), np.float64)
    for b in range(B):
        valid = idx[b] >= 0
        order = np.lexsort((idx[b][valid], d2[b][valid]))[:k]
        out_i[b] = idx[b][valid][order]
        out_d[b] = dist[b][valid][order]
        out_d2[b] = d2[b][valid][order]
    return out_i, out_d, out_d2


def gather_merge(li, ld, ld2, k, r0, world, group=None, device=None):
    """All-gather this rank's answers (local rows [B, k'], fp32 distances,
    FP64 squared distances; k' <= k) of every query and merge them: the global
    (rows, fp32 distances, FP64 squared distances) [B, k] on every rank.  Rows
    become global by adding r0, this shard's first row.  `device`: where the
    all-gather buffer lives (a CUDA device for NCCL; None: CPU, for gloo)."""
    import torch
    import torch.distributed as dist
    li = np.asarray(li, dtype=np.int64)
    B, kk = li.shape
    gi = np.full((B, k), -1, np.int64)
    gd = np.full((B, k), np.inf, np.float32)
    gd2 = np.full((B, k), np.inf, np.float64)
    gi[:, :kk] = li + r0
    gd[:, :kk] = np.asarray(ld, dtype=np.float32)
    gd2[:, :kk] = np.asarray(ld2, dtype=np.float64)
    # one buffer per query and rank: rows, fp32 distance bits and FP64 squared
    # distance bits packed as int64 columns (a single collective)
    pack = np.concatenate([gi, gd.view(np.int32).astype(np.int64), gd2.view(np.int64)], axis=1)
    t = torch.from_numpy(pack)
    if device is not None:
        t = t.to(device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    parts = [p.cpu().numpy() for p in parts]
    pi = [p[:, :k] for p in parts]
    pd = [p[:, k:2 * k].astype(np.int32).view(np.float32) for p in parts]
    pd2 = [np.ascontiguousarray(p[:, 2 * k:]).view(np.float64) for p in parts]
    return merge_knn(pi, pd, pd2, k)


def sharded_knn(local_search, Q, k, N, rank, world, group=None, device=None):
    """Exact k-NN of queries Q [B, n] over a collection sharded across the
    ranks of torch.distributed (`group`): local_search(Q, k) returns this
    rank's (local rows [B, k'], fp32 distances [B, k'], FP64 squared distances
    [B, k']) with k' = min(k, shard rows); every rank returns the merged global
    answer (rows, fp32 distances, FP64 squared distances)."""
    r0, r1 = shard_range(N, rank, world)
    li, ld, ld2 = local_search(Q, min(k, r1 - r0))
    return gather_merge(li, ld, ld2, k, r0, world, group=group, device=device)
