"""Exact k-NN over a collection split across ranks (one GPU per rank).

The collection shards by contiguous ranges of series (every series is summarised and
searched independently of the others, Section III), so each rank builds an index
over its range with no communication and answers every query over it. The one
exchange is an all-gather of each rank's k best per query, which are merged by
(FP64 squared distance, collection id): the same order the single-index answer uses,
so the merged answer equals the answer over the whole collection.
"""
import numpy as np


def merge_topk(ids_parts, d64_parts, k):
    """Merges per-shard answers. ids_parts / d64_parts: sequences of [nq, k_s] arrays
    (collection ids, FP64 squared distances). Returns (ids [nq, k], d64 [nq, k])
    ordered by (d64, id)."""
    ids = np.concatenate([np.asarray(p, dtype=np.int64) for p in ids_parts], axis=1)
    d64 = np.concatenate([np.asarray(p, dtype=np.float64) for p in d64_parts], axis=1)
    out_i = np.empty((ids.shape[0], k), dtype=np.int64)
    out_d = np.empty((ids.shape[0], k), dtype=np.float64)
    for q in range(ids.shape[0]):
        order = np.lexsort((ids[q], d64[q]))[:k]
        out_i[q], out_d[q] = ids[q, order], d64[q, order]
    return out_i, out_d


def gather_merge(ids, d64, k, group=None):
    """All-gathers this rank's (ids, d64) [nq, k] over torch.distributed and merges."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    ti = torch.as_tensor(np.ascontiguousarray(ids, dtype=np.int64))
    td = torch.as_tensor(np.ascontiguousarray(d64, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        ti, td = ti.cuda(), td.cuda()
    gi = [torch.empty_like(ti) for _ in range(world)]
    gd = [torch.empty_like(td) for _ in range(world)]
    dist.all_gather(gi, ti, group=group)
    dist.all_gather(gd, td, group=group)
    return merge_topk([g.cpu().numpy() for g in gi], [g.cpu().numpy() for g in gd], k)


def sharded_knn(index, queries, k, first_id, group=None, window=None):
    """k-NN over the whole sharded collection: this rank's answer over its index
    (collection ids offset by first_id), gathered and merged across the group.
    window=None: Euclidean (msi_knn_ex); an int: DTW with that warping window
    (msi_knn_dtw), whose FP64 DTW^2 merges the same way.
    Returns (ids int64 [nq, k], dists float32 [nq, k], d64 [nq, k])."""
    from . import msi_knn_dtw, msi_knn_ex
    if window is None:
        ids, _, d64 = msi_knn_ex(index, queries, k)
    else:
        ids, _, d64 = msi_knn_dtw(index, queries, k, window=window)
    if hasattr(ids, "cpu"):
        ids, d64 = ids.cpu().numpy(), d64.cpu().numpy()
    mi, md = gather_merge(ids + first_id, d64, k, group)
    return mi, np.sqrt(md).astype(np.float32), md
