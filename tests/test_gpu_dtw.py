"""DTW search on the GPU (msi_knn_dtw) against the oracle's FP64 DTW scan: the same
ids, the same FP64 DTW^2 bit for bit, the fp32 distance its rounding; over several
shapes (several leaves and blocks, a ragged last leaf, a length that is not a
multiple of 4), windows from 0 (the Euclidean distance) to unconstrained, k from 1
to past the warp-level top-k, both storage modes, an index with bounded query
slots, exact ties and constant series."""
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


def _check(msi, ix, X, Q, k, r, Z=None):
    ids, dists, d64 = msi.msi_knn_dtw(ix, Q, k, window=r)
    if Z is None:
        Z = oracle.summarise(X, ix.segments, 256)[0]
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], k, min(r, X.shape[1] - 1))
        assert np.array_equal(ids[i], oid), f"query {i}, k={k}, r={r}: {ids[i][:8]} vs {oid[:8]}"
        assert np.array_equal(d64[i], od2), f"query {i}, k={k}, r={r}: FP64 DTW differs"
        assert np.array_equal(dists[i], np.sqrt(od2).astype(np.float32))
    return ids, d64


SHAPES = [  # n, len, segments, leaf capacity
    (3000, 64, 16, 100),
    (5000, 128, 16, 300),
    (4000, 256, 16, 2000),
    (2500, 90, 10, 64),
]


@pytest.mark.parametrize("n,length,segs,cap", SHAPES)
def test_dtw_matches_oracle(msi, n, length, segs, cap):
    X = datagen.walks(301, 0, n, length)
    Z = oracle.summarise(X, segs, 256)[0]
    ix = msi.msi_build(X, segments=segs, leaf_capacity=cap)
    Q = np.concatenate([datagen.paper_queries(n, length, count=4, data_seed=301), X[[7]]])
    for r in (0, length // 10, length - 1):
        for k in (1, 5):
            _check(msi, ix, X, Q, k, r, Z)
    _check(msi, ix, X, Q[:2], 40, length // 10, Z)  # past the warp-level top-k
    ids, d64 = _check(msi, ix, X, Q[-1:], 1, length // 10, Z)
    assert ids[0, 0] == 7 and d64[0, 0] == 0.0
    ix.close()


def test_window_zero_is_the_euclidean_answer(msi):
    n, length = 4000, 128
    X = datagen.walks(302, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=100)
    Q = datagen.paper_queries(n, length, count=6, data_seed=302)
    ids_d, _, d64_d = msi.msi_knn_dtw(ix, Q, 3, window=0)
    ids_e, _, d64_e = msi.msi_knn_ex(ix, Q, 3)
    assert np.array_equal(ids_d, ids_e)
    np.testing.assert_allclose(d64_d, d64_e, rtol=1e-12)
    ix.close()


def test_window_past_the_length_is_unconstrained(msi):
    n, length = 1500, 64
    X = datagen.walks(303, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=50)
    Q = datagen.paper_queries(n, length, count=3, data_seed=303)
    a = msi.msi_knn_dtw(ix, Q, 4, window=length - 1)
    b = msi.msi_knn_dtw(ix, Q, 4, window=10 * length)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    ix.close()


def test_dtw_borrowed_device_collection(msi):
    import torch
    n, length = 6000, 256
    X = datagen.walks(304, 0, n, length)
    Xd = torch.from_numpy(X).cuda()
    ix = msi.msi_build(Xd, segments=16, leaf_capacity=200, flags=msi.MSI_BUILD_BORROW)
    Q = np.concatenate([datagen.paper_queries(n, length, count=4, data_seed=304), X[[123]]])
    Qd = torch.from_numpy(Q).cuda()
    ids, dists, d64 = msi.msi_knn_dtw(ix, Qd, 3, window=25)
    torch.cuda.synchronize()
    Z = oracle.summarise(X, 16, 256)[0]
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], 3, 25)
        assert np.array_equal(ids[i].cpu().numpy(), oid)
        assert np.array_equal(d64[i].cpu().numpy(), od2)
    ix.close()


def test_dtw_ties_constant_series_and_slots(msi):
    """Exact ties go to the lowest id; constant series (z = 0) are ordinary members;
    an index built with small query slots answers DTW queries exactly (they run on
    its full workspace)."""
    n, length = 5000, 128
    X = datagen.walks(305, 0, n, length)
    X[1000:1300] = X[999]        # 301 identical series
    X[4000:4010] = 3.5           # constant series
    Z = oracle.summarise(X, 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(n, length, count=5, data_seed=305), X[[999, 4003]]])
    ix = msi.msi_build(X, segments=16, leaf_capacity=100, query_slots=3, slot_capacity=256)
    for k in (1, 5, 32):
        ids, d64 = _check(msi, ix, X, Q, k, 12, Z)
        assert list(ids[5][:min(k, 5)]) == [999, 1000, 1001, 1002, 1003][:min(k, 5)]
        assert list(ids[6][:min(k, 5)]) == [4000, 4001, 4002, 4003, 4004][:min(k, 5)]
    ix.close()


def test_dtw_mixed_shapes(msi):
    n, length = 4000, 256
    X = datagen.mixed(306, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    ix = msi.msi_build(X, segments=16, leaf_capacity=150)
    Q = datagen.mixed_queries(count=5, length=length, query_seed=307)
    for k in (1, 10):
        _check(msi, ix, X, Q, k, 25, Z)
    ix.close()


def test_dtw_k_equals_n_full_order(msi):
    n, length = 300, 64
    X = datagen.walks(308, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=20)
    Q = datagen.paper_queries(n, length, count=2, data_seed=308)
    _check(msi, ix, X, Q, n, 6)
    ix.close()


def test_dtw_launch_count(msi):
    n, length = 2000, 64
    X = datagen.walks(309, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=50, query_slots=1)
    Q = datagen.paper_queries(n, length, count=2, data_seed=309)
    msi.msi_query_stats_get(ix, reset=True)
    msi.msi_knn_dtw(ix, Q, 1, window=6)
    assert msi.msi_query_stats_get(ix)["kernel_launches"] == 2 * 10
    msi.msi_knn_dtw(ix, Q[:1], 4, window=6)
    assert msi.msi_query_stats_get(ix)["kernel_launches"] == 2 * 10 + 12
    ix.close()


@pytest.mark.parametrize("n,length,segs,card,cap", [(4000, 256, 8, 16, 30), (1500, 60, 4, 4, 20)])
def test_dtw_small_cardinalities(msi, n, length, segs, card, cap):
    """Cardinalities below 32 (the coarse 5-bit tables then hold every symbol) and few
    segments, under DTW."""
    X = datagen.walks(310, 0, n, length)
    Z = oracle.summarise(X, segs, card)[0]
    ix = msi.msi_build(X, segments=segs, cardinality=card, leaf_capacity=cap)
    Q = np.concatenate([datagen.paper_queries(n, length, count=4, data_seed=310), X[[11]]])
    for k in (1, 6):
        ids, dists, d64 = msi.msi_knn_dtw(ix, Q, k, window=length // 10)
        for i, q in enumerate(Q):
            oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], k, length // 10)
            assert np.array_equal(ids[i], oid) and np.array_equal(d64[i], od2), (k, i)
    ix.close()


@pytest.mark.parametrize("n,length,cap", [(1200, 1024, 100), (2000, 512, 80)])
def test_dtw_long_series(msi, n, length, cap):
    """Long rows (screened from registers up to 1024 points) against the oracle."""
    X = datagen.walks(311, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    ix = msi.msi_build(X, segments=16, leaf_capacity=cap)
    Q = np.concatenate([datagen.paper_queries(n, length, count=2, data_seed=311), X[[5]]])
    ids, _, d64 = msi.msi_knn_dtw(ix, Q, 3, window=length // 10)
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], 3, length // 10)
        assert np.array_equal(ids[i], oid) and np.array_equal(d64[i], od2), i
    ix.close()
