"""Saved and loaded indexes (msi_index_save / msi_index_load): the loaded index holds
the same arrays and gives the same answers (Euclidean and DTW) as the one that was
saved, for an owned and for a borrowed collection; damaged files are rejected."""
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


def _same_index(msi, a, b):
    ea, eb = msi.msi_index_export(a), msi.msi_index_export(b)
    for key in ea:
        assert np.array_equal(ea[key], eb[key]), key


def test_owned_collection_round_trip(msi, tmp_path):
    n, length = 7000, 256
    X = datagen.walks(401, 0, n, length)
    ix = msi.msi_build(X, segments=16, leaf_capacity=300)
    Q = datagen.paper_queries(n, length, count=8, data_seed=401)
    ids_a, d_a = msi.msi_knn(ix, Q, 5)
    dtw_a = msi.msi_knn_dtw(ix, Q[:3], 3)
    path = str(tmp_path / "owned.idx")
    msi.msi_index_save(ix, path)
    jx = msi.msi_index_load(path, query_slots=2)
    _same_index(msi, ix, jx)
    ids_b, d_b = msi.msi_knn(jx, Q, 5)
    assert np.array_equal(ids_a, ids_b) and np.array_equal(d_a, d_b)
    dtw_b = msi.msi_knn_dtw(jx, Q[:3], 3)
    assert np.array_equal(dtw_a[0], dtw_b[0]) and np.array_equal(dtw_a[2], dtw_b[2])
    Z = oracle.summarise(X, 16, 256)[0]
    for i, q in enumerate(Q):
        assert np.array_equal(ids_b[i], oracle.knn_scan(Z, oracle.znorm(q)[0], 5)[0])
    ix.close()
    jx.close()


def test_borrowed_collection_round_trip_and_damage(msi, tmp_path):
    import torch
    n, length = 9000, 128
    X = datagen.walks(402, 0, n, length)
    Xd = torch.from_numpy(X).cuda()
    ix = msi.msi_build(Xd, segments=16, leaf_capacity=200, flags=msi.MSI_BUILD_BORROW)
    Q = datagen.paper_queries(n, length, count=6, data_seed=402)
    ids_a, d_a = msi.msi_knn(ix, Q, 3)
    path = tmp_path / "borrowed.idx"
    msi.msi_index_save(ix, str(path))
    with pytest.raises(msi.MsiError):  # the collection is not in the file
        msi.msi_index_load(str(path))
    jx = msi.msi_index_load(str(path), series=Xd)
    _same_index(msi, ix, jx)
    ids_b, d_b = msi.msi_knn(jx, Q, 3)
    assert np.array_equal(ids_a, ids_b) and np.array_equal(d_a, d_b)
    jx.close()
    # one flipped byte inside the SAX words: the checksum catches it
    raw = bytearray(path.read_bytes())
    raw[112 + 16 * 17 + 3] ^= 0x40
    bad = tmp_path / "bad.idx"
    bad.write_bytes(bytes(raw))
    with pytest.raises(msi.MsiError, match="checksum"):
        msi.msi_index_load(str(bad), series=Xd)
    bad.write_bytes(bytes(raw[:-8]))
    with pytest.raises(msi.MsiError, match="truncated"):
        msi.msi_index_load(str(bad), series=Xd)
    ix.close()
