"""Pins of the oracle's DTW search (Section IV, "MESSI with DTW") to facts outside
the oracle: hand-worked grids, brute force over every warping path, the Euclidean
special case, the closed form of the envelope on monotone series, and the chain of
lower bounds (PAA envelope <= LB_Keogh <= DTW)."""
import itertools

import numpy as np
import pytest

import datagen
import oracle


def _paths_min(a, b, r):
    """Brute force: the cheapest monotone warping path from (0, 0) to (n-1, n-1)
    with steps (1, 0), (0, 1), (1, 1) inside |i - j| <= r."""
    n = len(a)
    best = np.inf

    def walk(i, j, acc):
        nonlocal best
        acc += (float(a[i]) - float(b[j])) ** 2
        if acc >= best:
            return
        if i == n - 1 and j == n - 1:
            best = acc
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            ii, jj = i + di, j + dj
            if ii < n and jj < n and abs(ii - jj) <= r:
                walk(ii, jj, acc)

    walk(0, 0, 0.0)
    return best


def test_hand_worked_grids():
    # a warp of one step absorbs the shift completely
    assert oracle.dtw_sq([0, 0, 1, 2], [0, 1, 2, 2], 1) == 0.0
    assert oracle.dtw_sq([0, 0, 1, 2], [0, 1, 2, 2], 0) == 2.0
    # a = 1 2 3, b = 2 3 4: D(0,0) = 1, D(1,0) = 1, D(2,1) = 1, D(2,2) = 1 + 1 = 2
    assert oracle.dtw_sq([1, 2, 3], [2, 3, 4], 2) == 2.0
    assert oracle.dtw_sq([1, 2, 3], [2, 3, 4], 1) == 2.0
    assert oracle.dtw_sq([1, 2, 3], [2, 3, 4], 0) == 3.0
    assert oracle.dtw_sq([5.0], [2.0], 0) == 9.0


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_brute_force_over_warping_paths(n):
    rng = np.random.default_rng(n)
    for _ in range(12):
        a = rng.standard_normal(n).astype(np.float32)
        b = rng.standard_normal(n).astype(np.float32)
        for r in range(n):
            want = _paths_min(a, b, r)
            assert oracle.dtw_sq(a, b, r) == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_zero_window_is_squared_euclidean():
    X = datagen.walks(71, 0, 6, 256)
    for i in range(5):
        za, zb = oracle.znorm(X[i])[0], oracle.znorm(X[i + 1])[0]
        assert oracle.dtw_sq(za, zb, 0) == pytest.approx(oracle.sqdist(za, zb), rel=1e-12)


def test_symmetric_and_monotone_in_window():
    X = datagen.walks(72, 0, 4, 128)
    a, b = oracle.znorm(X[0])[0], oracle.znorm(X[1])[0]
    prev = np.inf
    for r in (0, 1, 2, 5, 12, 40, 127):
        d = oracle.dtw_sq(a, b, r)
        assert d == oracle.dtw_sq(b, a, r)
        assert d <= prev
        prev = d
    assert oracle.dtw_sq(a, a, 12) == 0.0


def test_envelope_closed_form_on_monotone_series():
    q = np.arange(20, dtype=np.float32) * 0.5
    for r in (0, 1, 3, 19):
        U, L = oracle.envelope(q, r)
        idx = np.arange(20)
        assert np.array_equal(U, q[np.minimum(idx + r, 19)])
        assert np.array_equal(L, q[np.maximum(idx - r, 0)])


def test_lower_bound_chain():
    """PAA-envelope mindist <= LB_Keogh <= DTW on random series and their own words."""
    n, w, c = 64, 16, 256
    X = datagen.walks(73, 0, 300, n)
    Z, _, W, _ = oracle.summarise(X, w, c)
    for r in (0, 2, 6, 63):
        for qi in range(0, 300, 37):
            zq = Z[qi]
            U, L = oracle.envelope(zq, r)
            Uh, Lh = oracle.paa_envelope(U, L, w)
            for i in range(0, 300, 7):
                d = oracle.dtw_sq(Z[i], zq, r)
                lbk = oracle.lb_keogh(U, L, Z[i])
                assert lbk <= d * (1 + 1e-12) + 1e-12
                # the word's region holds the fp32 PAA, which can sit an ulp outside
                # the exact mean: a small absolute slack
                assert oracle.mindist_env(Uh, Lh, W[i], W[i], n, c) <= np.sqrt(lbk) + 1e-5


def test_envelope_mindist_reduces_to_paa_mindist():
    """At r = 0 a query constant on every segment has Uh = Lh = its PAA."""
    n, w, c = 64, 16, 256
    rng = np.random.default_rng(5)
    q = np.repeat(rng.standard_normal(w), n // w).astype(np.float32)
    U, L = oracle.envelope(q, 0)
    Uh, Lh = oracle.paa_envelope(U, L, w)
    assert np.array_equal(Uh, Lh)
    assert np.array_equal(Uh, oracle.paa64(q, w))
    for _ in range(20):
        lo = rng.integers(0, 256, w).astype(np.uint8)
        hi = np.maximum(lo, rng.integers(0, 256, w)).astype(np.uint8)
        assert oracle.mindist_env(Uh, Lh, lo, hi, n, c) == oracle.mindist(Uh, lo, hi, n, c)


def test_scan_is_brute_force_with_ties_and_self_match():
    n, N, k = 32, 300, 6
    X = datagen.walks(74, 0, N, n)
    X[200] = X[17]  # a duplicate: a tie that goes to the lower id
    Z = oracle.summarise(X, 16, 256)[0]
    for r in (0, 3, 31):
        for q in (Z[17], Z[5], oracle.znorm(datagen.walks(75, 0, 1, n)[0])[0]):
            d = np.array([oracle.dtw_sq(Z[i], q, r) for i in range(N)])
            order = np.lexsort((np.arange(N), d))[:k]
            ids, d2 = oracle.knn_scan_dtw(Z, q, k, r)
            assert np.array_equal(ids, order)
            assert np.array_equal(d2, d[order])
        ids, d2 = oracle.knn_scan_dtw(Z, Z[17], 2, r)
        assert list(ids) == [17, 200] and list(d2) == [0.0, 0.0]


@pytest.mark.parametrize("n,r", [(64, 6), (128, 12), (128, 0)])
def test_index_search_equals_scan(n, r):
    N = 3000
    X = datagen.walks(76, 0, N, n)
    Z, _, W, _ = oracle.summarise(X, 16, 256)
    Q = datagen.paper_queries(N, n, count=6, data_seed=76)
    for q in Q:
        zq = oracle.znorm(q)[0]
        for k in (1, 7):
            ids_i, d_i, real = oracle.knn_index_dtw(Z, W, zq, k, r, cap=100)
            ids_s, d_s = oracle.knn_scan_dtw(Z, zq, k, r)
            assert np.array_equal(ids_i, ids_s)
            assert np.array_equal(d_i, d_s)
            assert real <= N
