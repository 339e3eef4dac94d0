"""The balanced split policy (MSI_BUILD_BALANCED_SPLIT, Section II-B: a node above
capacity splits on the segment whose next symbol bit divides its members most
evenly). The leaves must be exactly those of a plain restatement of the policy in
this file (root fan-out on the first bit of every segment in interleaved-key order,
then per node the most balanced open segment, lowest segment on ties, a stable
partition on its bit, pieces of the capacity once no bit is left), and searches on
such an index must give the oracle's answers, Euclidean and DTW, also after a save
and load."""
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


def _keys(W, bits):
    """First 64 bits of the interleaved key: bit planes from the most significant,
    segment 0 first within a plane."""
    n, w = W.shape
    keys = np.zeros(n, dtype=np.uint64)
    used = 0
    for plane in range(bits - 1, -1, -1):
        for j in range(w):
            if used == 64:
                return keys
            keys = (keys << np.uint64(1)) | ((W[:, j].astype(np.uint64) >> np.uint64(plane)) & np.uint64(1))
            used += 1
    return keys << np.uint64(64 - used)


def reference_leaves(W, bits, cap):
    """(perm, leaf_begin) of the balanced policy, written out on the host."""
    n, w = W.shape
    keys = _keys(W, bits)
    order = np.lexsort((np.arange(n), keys))
    prefix = keys[order] >> np.uint64(64 - w)
    perm, begins = [], []

    def split(ids, depth):
        size = len(ids)
        open_ = [j for j in range(w) if depth[j] < bits]
        if size <= cap or not open_:
            for p in range(0, size, cap):
                begins.append(len(perm) + p)
            perm.extend(ids)
            return
        best, gap = None, None
        for j in open_:
            ones = int(((W[ids, j] >> (bits - 1 - depth[j])) & 1).sum())
            g = abs(2 * ones - size)
            if best is None or g < gap:
                best, gap = j, g
        bit = (W[ids, best] >> (bits - 1 - depth[best])) & 1
        d2 = list(depth)
        d2[best] += 1
        for side in (0, 1):
            part = ids[bit == side]
            if len(part):
                split(part, d2)

    start = 0
    for i in range(1, n + 1):
        if i == n or prefix[i] != prefix[start]:
            split(order[start:i], [1] * w)
            start = i
    return np.array(perm, dtype=np.uint32), np.array(begins + [n], dtype=np.uint32)


SHAPES = [  # n, len, segments, leaf capacity
    (6000, 256, 16, 64),
    (5000, 128, 16, 300),
    (3000, 64, 8, 50),
    (2500, 90, 10, 64),
]


@pytest.mark.parametrize("n,length,segs,cap", SHAPES)
def test_leaves_follow_the_policy_and_answers_are_exact(msi, n, length, segs, cap):
    X = datagen.walks(501, 0, n, length)
    X[100:400] = X[99]  # 301 identical series: a node no bit can split
    Z, _, W, _ = oracle.summarise(X, segs, 256)
    ix = msi.msi_build(X, segments=segs, leaf_capacity=cap, flags=msi.MSI_BUILD_BALANCED_SPLIT)
    ex = msi.msi_index_export(ix)
    perm, begins = reference_leaves(W, 8, cap)
    assert np.array_equal(ex["perm"], perm)
    assert np.array_equal(ex["leaf_begin"], begins)
    Q = np.concatenate([datagen.paper_queries(n, length, count=5, data_seed=501), X[[99, 2000]]])
    for k in (1, 10, 100):
        ids, d = msi.msi_knn(ix, Q, k)
        for i, q in enumerate(Q):
            oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
            assert np.array_equal(ids[i], oid), (k, i)
    ids, _, d64 = msi.msi_knn_dtw(ix, Q[:3], 3, window=length // 10)
    for i, q in enumerate(Q[:3]):
        oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], 3, length // 10)
        assert np.array_equal(ids[i], oid) and np.array_equal(d64[i], od2)
    ix.close()


def test_balanced_index_round_trip(msi, tmp_path):
    n, length = 8000, 128
    X = datagen.walks(502, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=100, flags=msi.MSI_BUILD_BALANCED_SPLIT)
    Q = datagen.paper_queries(n, length, count=6, data_seed=502)
    a = msi.msi_knn(ix, Q, 4)
    path = str(tmp_path / "balanced.idx")
    msi.msi_index_save(ix, path)
    jx = msi.msi_index_load(path)
    b = msi.msi_knn(jx, Q, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert msi.msi_index_info_get(jx)["flags"] & msi.MSI_BUILD_BALANCED_SPLIT
    ix.close()
    jx.close()
