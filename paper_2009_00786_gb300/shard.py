"""Exact k-NN over a collection split across ranks (one GPU per rank).

The collection shards by contiguous ranges of series (every series is summarised and
searched independently of the others, Section III), so each rank builds an index
over its range with no communication and answers every query over it. The one
exchange is an all-gather of each rank's k best per query, which the library merges
on the GPU (msi_merge_topk) by (FP64 squared distance, collection id): the same order
the single-index answer uses, so the merged answer equals the answer over the whole
collection.
"""
import numpy as np


def merge_topk(ids_parts, d64_parts, k, stream=None):
    """Merges per-shard answers with msi_merge_topk. ids_parts / d64_parts: sequences
    of [nq, k_s] arrays (collection ids, FP64 squared distances; numpy or torch, each
    row sorted as msi_knn_ex returns it). Returns (ids [nq, k], d64 [nq, k]) ordered
    by (d64, id), as numpy arrays."""
    from . import msi_merge_topk
    if all(hasattr(p, "data_ptr") for p in ids_parts):
        import torch
        ids = torch.stack([p.to(torch.int64) for p in ids_parts]).contiguous()
        d64 = torch.stack([p.to(torch.float64) for p in d64_parts]).contiguous()
    else:
        ids = np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.int64) for p in ids_parts]))
        d64 = np.ascontiguousarray(np.stack([np.asarray(p, dtype=np.float64) for p in d64_parts]))
    mi, _, md = msi_merge_topk(ids, d64, k, stream)
    if hasattr(mi, "cpu"):
        mi, md = mi.cpu().numpy(), md.cpu().numpy()
    return mi, md


def gather_merge(ids, d64, k, group=None, stream=None, merge=None):
    """All-gathers this rank's (ids, d64) [nq, k] over torch.distributed and merges
    them with msi_merge_topk on this rank's GPU (`merge` replaces it: a callable
    (ids [parts, nq, k_in], d64 [parts, nq, k_in], k) -> (ids, dists, d64), used by
    the host-only tests of the exchange). Returns (ids int64 [nq, k], dists float32
    [nq, k], d64 [nq, k])."""
    import torch
    import torch.distributed as dist

    from . import msi_merge_topk
    world = dist.get_world_size(group)
    ti = ids if hasattr(ids, "data_ptr") else torch.as_tensor(np.ascontiguousarray(ids, dtype=np.int64))
    td = d64 if hasattr(d64, "data_ptr") else torch.as_tensor(np.ascontiguousarray(d64, dtype=np.float64))
    nccl = dist.get_backend(group) == "nccl"
    ti, td = (ti.cuda(), td.cuda()) if nccl else (ti.cpu(), td.cpu())
    gi = torch.empty((world,) + tuple(ti.shape), dtype=torch.int64, device=ti.device)
    gd = torch.empty((world,) + tuple(td.shape), dtype=torch.float64, device=td.device)
    dist.all_gather(list(gi.unbind(0)), ti.contiguous(), group=group)
    dist.all_gather(list(gd.unbind(0)), td.contiguous(), group=group)
    if merge is not None:
        return merge(gi, gd, k)
    if not nccl:  # the merge runs on this rank's GPU
        gi, gd = gi.cuda(), gd.cuda()
    return msi_merge_topk(gi, gd, k, stream)


def sharded_knn(index, queries, k, first_id, group=None, window=None, stream=None):
    """k-NN over the whole sharded collection: this rank's answer over its index
    (collection ids offset by first_id), gathered and merged across the group.
    window=None: Euclidean (msi_knn_ex); an int: DTW with that warping window
    (msi_knn_dtw), whose FP64 DTW^2 merges the same way.
    Returns (ids int64 [nq, k], dists float32 [nq, k], d64 [nq, k]) on the device of
    the merge."""
    from . import msi_knn_dtw, msi_knn_ex
    if window is None:
        ids, _, d64 = msi_knn_ex(index, queries, k, stream)
    else:
        ids, _, d64 = msi_knn_dtw(index, queries, k, window=window, stream=stream)
    return gather_merge(ids + first_id, d64, k, group, stream)
