"""The multi-rank exchange on the CPU: two gloo ranks each answer the queries over
their half of the collection (with the oracle, as a GPU rank answers with its index)
and exchange them through paper_2009_00786_gb300.shard.gather_merge; the merged answer
must equal the oracle's answer over the whole collection, ties included. The library
merges on the GPU (msi_merge_topk, tested in test_gpu_multirank.py); here, with no
GPU, the merge step is the definition written out: all candidates sorted by
(distance, id), the first k kept."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle

N, LEN, K = 3000, 128, 7


def host_merge(gi, gd, k):
    """The k smallest of every part's candidates by (FP64 distance, id)."""
    ids = np.concatenate(list(gi.numpy()), axis=1)
    d64 = np.concatenate(list(gd.numpy()), axis=1)
    out_i = np.empty((ids.shape[0], k), dtype=np.int64)
    out_d = np.empty((ids.shape[0], k), dtype=np.float64)
    for q in range(ids.shape[0]):
        order = np.lexsort((ids[q], d64[q]))[:k]
        out_i[q], out_d[q] = ids[q, order], d64[q, order]
    return out_i, np.sqrt(out_d).astype(np.float32), out_d


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_dtw(rank, world, port, out_path):
    import torch.distributed as dist

    from paper_2009_00786_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = datagen.walks(62, 0, 1200, 64)
    X[1100] = X[20]  # a tie across the two shards
    per = 1200 // world
    first = rank * per
    Z = oracle.summarise(X[first:first + per], 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(1200, 64, count=4, data_seed=62), X[[20]]])
    ids, d2 = [], []
    for q in Q:
        i, d = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], K, 6)
        ids.append(i + first)
        d2.append(d)
    mi, _, md = shard.gather_merge(np.array(ids), np.array(d2), K, merge=host_merge)
    if rank == 0:
        np.savez(out_path, ids=mi, d2=md)
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_dtw_answers(tmp_path):
    """The same exchange under DTW: per-rank FP64 DTW^2 answers merge into the
    whole-collection DTW answer."""
    try:
        import __graft_entry__
        __graft_entry__.build()
    except Exception as e:
        pytest.skip(f"library build unavailable: {e}")
    import torch.multiprocessing as mp
    out = str(tmp_path / "merged_dtw.npz")
    mp.start_processes(_rank_dtw, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    X = datagen.walks(62, 0, 1200, 64)
    X[1100] = X[20]
    Z = oracle.summarise(X, 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(1200, 64, count=4, data_seed=62), X[[20]]])
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], K, 6)
        assert np.array_equal(got["ids"][i], oid)
        assert np.array_equal(got["d2"][i], od2)
    assert list(got["ids"][-1][:2]) == [20, 1100]


def _rank(rank, world, port, out_path):
    import torch.distributed as dist

    from paper_2009_00786_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = datagen.walks(61, 0, N, LEN)
    X[2500] = X[10]  # a tie across the two shards
    per = N // world
    first = rank * per
    Z = oracle.summarise(X[first:first + per], 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(N, LEN, count=6, data_seed=61), X[[10]]])
    ids, d2 = [], []
    for q in Q:
        i, d = oracle.knn_scan(Z, oracle.znorm(q)[0], K)
        ids.append(i + first)
        d2.append(d)
    mi, _, md = shard.gather_merge(np.array(ids), np.array(d2), K, merge=host_merge)
    if rank == 0:
        np.savez(out_path, ids=mi, d2=md)
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_whole_answer(tmp_path):
    try:
        import __graft_entry__
        __graft_entry__.build()
    except Exception as e:  # the package needs its library only to import
        pytest.skip(f"library build unavailable: {e}")
    import torch.multiprocessing as mp
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    X = datagen.walks(61, 0, N, LEN)
    X[2500] = X[10]
    Z = oracle.summarise(X, 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(N, LEN, count=6, data_seed=61), X[[10]]])
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], K)
        assert np.array_equal(got["ids"][i], oid)
        assert np.array_equal(got["d2"][i], od2)
    assert list(got["ids"][-1][:2]) == [10, 2500]
