"""The fine PAA bound (default; MSI_BUILD_NO_FINE_BOUND turns it off): the index keeps
each series' means over wf equal segments as fp16 (a PAA, Section II-B, over finer
segments than the iSAX word), and the series filter bounds every series that passes
the iSAX bound by them before its row is read. The stored means must be the fp16
roundings of the z-normalised series' segment means, the segment count must follow
the documented rule, and answers must be the oracle's with the bound on and off,
Euclidean and DTW, with fewer rows read when it is on."""
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


def expected_wf(length, w):
    for wf in (64, 32, 16, 8):
        sf = length // wf
        if length % wf == 0 and sf & (sf - 1) == 0 and wf > w:
            return wf
    return 0


SHAPES = [  # n, len, segments, expected fine segments
    (3000, 256, 16, 64),   # 4-point segments
    (2000, 128, 16, 64),   # 2-point segments
    (1500, 64, 8, 64),     # the series itself, in fp16
    (1200, 1024, 16, 64),  # 16-point segments
    (1000, 512, 16, 64),
    (700, 256, 8, 64),
    (600, 32, 16, 32),     # one point per fine segment
    (900, 96, 8, 0),       # no power-of-two segment length
    (800, 384, 16, 0),
]


@pytest.mark.parametrize("n,length,segs,wf", SHAPES)
def test_fine_means_are_fp16_segment_means(msi, n, length, segs, wf):
    assert expected_wf(length, segs) == wf
    X = datagen.walks(601, 0, n, length)
    X[5] = 3.0          # a constant series: all means 0
    X[6] = 0.0
    X[6, 7] = 1.0       # one spike: the largest z a series of this length can hold
    ix = msi.msi_build(X, segments=segs, leaf_capacity=50)
    assert msi.msi_index_info_get(ix)["fine_segments"] == wf
    ex = msi.msi_index_export(ix, fine=True, znorm=True)
    if wf == 0:
        assert "fine" not in ex
        ix.close()
        return
    Z = oracle.summarise(X, segs, 256)[0]
    assert np.array_equal(ex["znorm"], Z)
    m = Z.astype(np.float64).reshape(n, wf, length // wf).mean(axis=2)
    h = ex["fine"].astype(np.float64)
    # round to nearest fp16 of an fp32 mean: within half an fp16 ulp, plus the fp32
    # rounding of the mean itself
    assert np.all(np.abs(h - m) <= np.abs(h) * 2.0 ** -11 + 2.0 ** -25 + 1e-6 * np.maximum(1.0, np.abs(m)))
    assert np.all(h[5] == 0.0)
    ix.close()


@pytest.mark.parametrize("length", [256, 128, 64])
def test_answers_match_oracle_and_fewer_rows_are_read(msi, length):
    n = 20000
    X = datagen.walks(602, 0, n, length)
    Z = oracle.summarise(X, 16 if length > 64 else 8, 256)[0]
    Q = datagen.paper_queries(n, length, count=12, data_seed=602)
    segs = 16 if length > 64 else 8
    on = msi.msi_build(X, segments=segs, leaf_capacity=100)
    off = msi.msi_build(X, segments=segs, leaf_capacity=100, flags=msi.MSI_BUILD_NO_FINE_BOUND)
    assert msi.msi_index_info_get(off)["fine_segments"] == 0
    refined = {}
    for name, ix in (("on", on), ("off", off)):
        msi.msi_query_stats_get(ix, reset=True)
        for k in (1, 10):
            ids, d = msi.msi_knn(ix, Q, k)
            for i, q in enumerate(Q):
                oid, _ = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
                assert np.array_equal(ids[i], oid), (name, k, i)
        st = msi.msi_query_stats_get(ix)
        refined[name] = st["series_refined"]
        # the fine bound runs only on the index that keeps the fine PAA, and only on
        # series whose iSAX bound passed (so never more often than the words bounded)
        if name == "on":
            assert 0 < st["fine_bounded"] <= st["series_lower_bounded"]
            assert st["survivors"] <= st["fine_bounded"]
        else:
            assert st["fine_bounded"] == 0 and st["front_fine_bounded"] == 0
    assert refined["on"] < refined["off"], refined
    for name, ix in (("on", on), ("off", off)):
        ids, _, d64 = msi.msi_knn_dtw(ix, Q[:4], 3, window=length // 10)
        for i, q in enumerate(Q[:4]):
            oid, od2 = oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], 3, length // 10)
            assert np.array_equal(ids[i], oid) and np.array_equal(d64[i], od2), (name, i)
    on.close()
    off.close()


def test_fine_bound_survives_save_and_load(msi, tmp_path):
    n, length = 5000, 256
    X = datagen.walks(603, 0, n, length)
    Q = datagen.paper_queries(n, length, count=5, data_seed=603)
    for flags in (0, 4):
        ix = msi.msi_build(X, segments=16, leaf_capacity=64, flags=flags)
        a = msi.msi_knn(ix, Q, 3)
        path = str(tmp_path / f"fine{flags}.idx")
        msi.msi_index_save(ix, path)
        jx = msi.msi_index_load(path)
        assert msi.msi_index_info_get(jx)["fine_segments"] == (0 if flags else 64)
        b = msi.msi_knn(jx, Q, 3)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        if not flags:
            assert np.array_equal(msi.msi_index_export(ix, fine=True)["fine"].view(np.uint16),
                                  msi.msi_index_export(jx, fine=True)["fine"].view(np.uint16))
        ix.close()
        jx.close()
