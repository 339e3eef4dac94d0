"""The multi-rank path on real kernels. msi_merge_topk against the definition of the
merge (every candidate sorted by (FP64 distance, id), the first k kept); then two
processes that share cuda:0, each building an index over its half of a collection
with msi_build and answering with msi_knn_ex, exchange their answers over gloo and
merge them on the GPU: the merged answer must equal the oracle's answer over the
whole collection, a tie across the two halves included."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

N, LEN, K = 20000, 128, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _definition(ids, d64, k):
    ids = np.concatenate(list(ids), axis=1)
    d64 = np.concatenate(list(d64), axis=1)
    out_i = np.empty((ids.shape[0], k), dtype=np.int64)
    out_d = np.empty((ids.shape[0], k), dtype=np.float64)
    for q in range(ids.shape[0]):
        o = np.lexsort((ids[q], d64[q]))[:k]
        out_i[q], out_d[q] = ids[q, o], d64[q, o]
    return out_i, out_d


def test_merge_topk_on_the_gpu_equals_the_definition():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as msi
    rng = np.random.default_rng(3)
    parts, nq, kin = 4, 9, 12
    ids = np.empty((parts, nq, kin), dtype=np.int64)
    d64 = np.empty((parts, nq, kin), dtype=np.float64)
    for p in range(parts):
        for q in range(nq):
            d = np.sort(rng.integers(0, 20, size=kin).astype(np.float64) * 0.5)  # many exact ties
            i = np.sort(rng.choice(1000, size=kin, replace=False)) + 1000 * p  # distinct across parts
            o = np.lexsort((i, d))
            ids[p, q], d64[p, q] = i[o], d[o]
    for k in (1, 5, kin, parts * kin):
        want_i, want_d = _definition(ids, d64, k)
        for dev in (False, True):
            a = torch.from_numpy(ids).cuda() if dev else ids
            b = torch.from_numpy(d64).cuda() if dev else d64
            gi, gf, gd = msi.msi_merge_topk(a, b, k)
            if dev:
                torch.cuda.synchronize()
                gi, gf, gd = gi.cpu().numpy(), gf.cpu().numpy(), gd.cpu().numpy()
            assert np.array_equal(gi, want_i), (k, dev)
            assert np.array_equal(gd, want_d), (k, dev)
            assert np.array_equal(gf, np.sqrt(want_d).astype(np.float32)), (k, dev)
    with pytest.raises(msi.MsiError):
        msi.msi_merge_topk(ids, d64, parts * kin + 1)


def _collection():
    X = datagen.walks(61, 0, N, LEN)
    X[15000] = X[10]  # a tie across the two halves
    Q = np.concatenate([datagen.paper_queries(N, LEN, count=6, data_seed=61), X[[10]]])
    return X, Q


def _rank(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import paper_2009_00786_gb300 as msi
    from paper_2009_00786_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)  # both ranks share the one GPU; no kernel waits on the other's
    X, Q = _collection()
    per = N // world
    first = rank * per
    index = msi.msi_build(torch.from_numpy(X[first:first + per]).cuda(), segments=16, cardinality=256,
                          leaf_capacity=200)
    mi, md, m64 = shard.sharded_knn(index, torch.from_numpy(Q).cuda(), K, first)
    torch.cuda.synchronize()
    if rank == 0:
        np.savez(out_path, ids=mi.cpu().numpy(), d=md.cpu().numpy(), d64=m64.cpu().numpy())
    index.close()
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_merge_to_the_whole_answer(tmp_path):
    import torch.multiprocessing as mp

    import __graft_entry__
    __graft_entry__.build()
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    X, Q = _collection()
    Z = oracle.summarise(X, 16, 256)[0]
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], K)
        assert np.array_equal(got["ids"][i], oid), (i, got["ids"][i], oid)
        np.testing.assert_allclose(got["d64"][i], od2, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got["d"][i], np.sqrt(od2), rtol=1e-4, atol=1e-6)
    assert list(got["ids"][-1][:2]) == [10, 15000]
