"""The tensor-core filter of the batched chain (msi_schedule batch_dense = 1): one
streaming pass of tcgen05 TF32 dot products per pass of queries, a certified lower
bound per (series, query) pair, fp32 distances of the survivors and the FP64 re-check.
Its answers must be exactly the oracle's and those of the iSAX-pruned chain: borrowed
(raw) and owned (z-normalised) collections, random walks and the mixed shapes, series
lengths that fill several passes of queries or end inside a 32-point block, a ragged
last tile of series, exact ties, constant series and a constant query, k = 1 and 10,
and survivor lists too small for the first tiles (the query then runs again alone)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as m
    return m


CASES = [  # kind, borrowed, length, segments, n, queries
    ("walks", True, 256, 16, 40000 - 3, 20),
    ("mixed", False, 256, 16, 30000, 20),
    ("walks", False, 128, 16, 25000, 20),
    ("walks", True, 1024, 16, 6000, 40),   # 32 queries per pass: two passes
    ("walks", True, 100, 10, 9000, 12),    # the last 32-point block is partly past the series
]


@pytest.mark.parametrize("kind,borrow,length,w,n,nq", CASES)
def test_dense_filter_matches_oracle_and_pruned_chain(msi, kind, borrow, length, w, n, nq):
    import torch
    gen = datagen.mixed if kind == "mixed" else datagen.walks
    X = gen(71, 0, n, length)
    X[n - 2] = X[17]            # an exact tie, far apart in id
    X[5] = 3.0                  # two constant series: z = 0
    X[7] = -1.0
    Q = np.concatenate([datagen.walks(72, 0, nq - 3, length), X[[17, 300]] + 0.001 * datagen.walks(73, 0, 2, length),
                        np.full((1, length), 2.0, dtype=np.float32)])  # a constant query
    Z = oracle.summarise(X, w, 256)[0]
    src = torch.from_numpy(X).cuda() if borrow else X
    ix = msi.msi_build(src, segments=w, cardinality=256, leaf_capacity=300,
                       flags=msi.MSI_BUILD_BORROW if borrow else 0)
    Qd = torch.from_numpy(Q).cuda()
    for k in (1, 10):
        msi.msi_schedule_set(ix, batch_chain=1, batch_dense=0, batch_group=128)
        ids_p, d_p = msi.msi_knn(ix, Qd, k)
        msi.msi_schedule_set(ix, batch_chain=1, batch_dense=1, batch_group=128)
        msi.msi_query_stats_get(ix, reset=True)
        ids, d = msi.msi_knn(ix, Qd, k)
        st = msi.msi_query_stats_get(ix, reset=True)
        assert st["tc_pairs"] == n * nq, (st["tc_pairs"], n * nq)
        ids, d = ids.cpu().numpy(), d.cpu().numpy()
        assert np.array_equal(ids, ids_p.cpu().numpy()) and np.array_equal(d, d_p.cpu().numpy())
        for i, q in enumerate(Q):
            oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
            assert np.array_equal(ids[i], oid), (k, i, ids[i], oid)
            np.testing.assert_allclose(d[i], np.sqrt(od2), rtol=1e-4, atol=1e-6)
        assert ids[-1][0] == 5 and (k == 1 or ids[-1][1] == 7)  # constant query: constant series, lower id first
        assert ids[-3][0] == 17 and (k == 1 or ids[-3][1] == n - 2)
    ix.close()


def test_dense_filter_survivor_overflow_reruns(msi):
    """Survivor lists of 8 entries: the first tiles of the pass keep more pairs than
    that before the thresholds tighten, so queries overflow and run again alone; the
    answers stay the oracle's."""
    import torch
    n, length, nq = 20000, 256, 8
    X = datagen.walks(81, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    Q = datagen.paper_queries(n, length, count=nq, data_seed=81)
    ix = msi.msi_build(torch.from_numpy(X).cuda(), segments=16, leaf_capacity=200, flags=msi.MSI_BUILD_BORROW,
                       slot_capacity=8)
    msi.msi_schedule_set(ix, batch_chain=1, batch_dense=1, batch_group=8)
    msi.msi_query_stats_get(ix, reset=True)
    ids, d = msi.msi_knn(ix, torch.from_numpy(Q).cuda(), 3)
    st = msi.msi_query_stats_get(ix)
    assert st["overflow_reruns"] > 0
    for i, q in enumerate(Q):
        oid, _ = oracle.knn_scan(Z, oracle.znorm(q)[0], 3)
        assert np.array_equal(ids[i].cpu().numpy(), oid), i
    ix.close()
