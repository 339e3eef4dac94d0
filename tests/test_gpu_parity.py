"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances: SAX words, z-normalised values, thresholds, leaf structure and neighbour
ids bit-exact; distances within 1e-4 relative (they are FP64 results rounded to
float on both sides, so in practice equal).
"""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def msi():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as m
    return m


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


# (n, len, segments, cardinality, leaf capacity): several radix tiles and a ragged
# tail, both summarise paths (len a power-of-two multiple of 128, and not), scalar
# and vector distance paths, small words and alphabets.
CASES = [
    (20000, 256, 16, 256, 64),
    (5003, 128, 16, 256, 2000),
    (3001, 1024, 16, 256, 100),
    (2500, 96, 16, 256, 50),
    (4000, 256, 8, 16, 30),
    (1500, 60, 4, 4, 20),
    (777, 50, 5, 256, 10),
    (3333, 512, 16, 256, 100),   # two series per warp, segments of 32 points, odd n
    (2001, 256, 4, 64, 50),      # two series per warp, segments of 64 points
]
IDS = [f"n{c[0]}-len{c[1]}-w{c[2]}-c{c[3]}-cap{c[4]}" for c in CASES]

_cache = {}


def case_data(case):
    if case not in _cache:
        n, length, w, c, cap = case
        X = datagen.walks(100 + n, 0, n, length)
        Z, P, W, F = oracle.summarise(X, w, c)
        _cache[case] = (X, Z, W)
    return _cache[case]


def build(msi, X, case, mode="host", torch=None):
    n, length, w, c, cap = case
    if mode == "host":
        return msi.msi_build(X, segments=w, cardinality=c, leaf_capacity=cap)
    t = torch.from_numpy(X).cuda()
    if mode == "device":
        return msi.msi_build(t, segments=w, cardinality=c, leaf_capacity=cap)
    return msi.msi_build(t, segments=w, cardinality=c, leaf_capacity=cap, flags=msi.MSI_BUILD_BORROW)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_summaries_bit_exact(msi, case):
    n, length, w, c, cap = case
    X, Z, W = case_data(case)
    ix = build(msi, X, case)
    ex = msi.msi_index_export(ix, znorm=True)
    assert np.array_equal(ex["thresholds"], oracle.thresholds(c))
    assert np.array_equal(ex["znorm"].view(np.uint32), Z.view(np.uint32))
    bad = np.nonzero((ex["words"] != W).any(axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} words differ, first ids {bad[:5]}"


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_leaf_structure(msi, case):
    n, length, w, c, cap = case
    X, Z, W = case_data(case)
    ix = build(msi, X, case)
    ex = msi.msi_index_export(ix)
    lb, perm = ex["leaf_begin"].astype(np.int64), ex["perm"].astype(np.int64)
    assert lb[0] == 0 and lb[-1] == n and np.all(np.diff(lb) > 0)
    assert np.all(np.diff(lb) <= cap)
    assert np.array_equal(np.sort(perm), np.arange(n))
    bits = int(np.log2(c))
    Wl = W[perm]
    for l in range(len(lb) - 1):
        m = Wl[lb[l]:lb[l + 1]]
        assert np.array_equal(ex["env_lo"][l], m.min(axis=0))
        assert np.array_equal(ex["env_hi"][l], m.max(axis=0))
        # members of a leaf share their root subtree: the top bit of every symbol
        assert np.all((m >> (bits - 1)) == (m[0] >> (bits - 1)))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_knn_matches_oracle(msi, case):
    n, length, w, c, cap = case
    X, Z, W = case_data(case)
    ix = build(msi, X, case)
    Q = datagen.paper_queries(n, length, count=10, data_seed=100 + n, fresh_seed=7, pick_seed=8)
    for k in [1, 10, 100]:
        if k > n:
            continue
        ids, dists = msi.msi_knn(ix, Q, k)
        for i, q in enumerate(Q):
            oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
            assert np.array_equal(ids[i], oid), f"k={k} query {i}: {ids[i][:8]} vs {oid[:8]}"
            np.testing.assert_allclose(dists[i], np.sqrt(od2), rtol=RTOL, atol=1e-6)


def test_input_modes_agree(msi, torch):
    case = CASES[0]
    X, Z, W = case_data(case)
    Q = datagen.paper_queries(case[0], case[1], count=8, data_seed=100 + case[0])
    Qd = torch.from_numpy(Q).cuda()
    out = []
    for mode in ("host", "device", "borrow"):
        ix = build(msi, X, case, mode, torch)
        ids, d = msi.msi_knn(ix, Qd, 10)
        out.append((ids.cpu().numpy(), d.cpu().numpy()))
        ids_h, d_h = msi.msi_knn(ix, Q, 10)  # host queries and outputs
        assert np.array_equal(ids_h, out[-1][0]) and np.array_equal(d_h, out[-1][1])
    for ids, d in out[1:]:
        assert np.array_equal(ids, out[0][0]) and np.array_equal(d, out[0][1])


def test_stream_ordered_call(msi, torch):
    case = CASES[0]
    X, Z, W = case_data(case)
    Q = torch.from_numpy(datagen.paper_queries(case[0], case[1], count=5, data_seed=100 + case[0])).cuda()
    ix = build(msi, X, case)
    want = msi.msi_knn(ix, Q, 3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ids = torch.empty((5, 3), dtype=torch.int64, device="cuda")
        d = torch.empty((5, 3), dtype=torch.float32, device="cuda")
        msi.msi_knn(ix, Q, 3, ids, d, stream=s)
    s.synchronize()
    assert torch.equal(ids, want[0]) and torch.equal(d, want[1])


def test_edge_cases(msi):
    length = 128
    X = datagen.walks(3, 0, 300, length)
    # a single series
    ix = msi.msi_build(X[:1], segments=16)
    ids, d = msi.msi_knn(ix, X[:2], 1)
    assert list(ids[:, 0]) == [0, 0] and d[0, 0] == 0.0
    # k = n: the full order
    ix = msi.msi_build(X, segments=16, leaf_capacity=16)
    Z = oracle.summarise(X, 16, 256)[0]
    ids, d = msi.msi_knn(ix, X[5:6], 300)
    oid, od2 = oracle.knn_scan(Z, oracle.znorm(X[5])[0], 300)
    assert np.array_equal(ids[0], oid) and ids[0, 0] == 5
    # duplicates and constant series: ties go to the lowest id
    Xd = X.copy()
    Xd[200] = Xd[40]
    Xd[250] = Xd[40] * np.float32(3.0) + np.float32(1.0)  # same z-normalised shape
    Xd[10] = 7.0
    Xd[11] = -2.0
    ix = msi.msi_build(Xd, segments=16, leaf_capacity=8)
    ids, d = msi.msi_knn(ix, Xd[[200, 11]], 3)
    Zd = oracle.summarise(Xd, 16, 256)[0]
    for row, q in zip(ids, Xd[[200, 11]]):
        assert np.array_equal(row, oracle.knn_scan(Zd, oracle.znorm(q)[0], 3)[0])
    assert ids[0, 0] == 40 and ids[1, 0] == 10 and ids[1, 1] == 11  # constant query -> constant series
    # invalid inputs
    Xn = X.copy()
    Xn[17, 3] = np.nan
    with pytest.raises(msi.MsiError) as e:
        msi.msi_build(Xn, segments=16)
    assert e.value.status == msi.MSI_EINVAL and "series 17" in str(e.value)
    Qn = X[:2].copy()
    Qn[1, 0] = np.inf
    with pytest.raises(msi.MsiError):
        msi.msi_knn(ix, Qn, 1)
    for k in (0, 301, 2000):
        with pytest.raises(msi.MsiError):
            msi.msi_knn(ix, X[:1], k)
    ids, d = msi.msi_knn(ix, X[:0], 1)  # nq = 0
    assert ids.shape == (0, 1)


def test_lower_bounds_are_bounds(msi):
    case = (6000, 256, 16, 256, 64)
    X = datagen.walks(9, 0, case[0], 256)
    Z, _, W, _ = oracle.summarise(X, 16, 256)
    ix = msi.msi_build(X, segments=16, leaf_capacity=64)
    ex = msi.msi_index_export(ix)
    perm, lb = ex["perm"].astype(np.int64), ex["leaf_begin"].astype(np.int64)
    for q in datagen.walks(10, 0, 3, 256):
        zq = oracle.znorm(q)[0]
        s_lb, l_lb = msi.msi_lower_bounds(ix, q)
        true = np.sqrt(((Z.astype(np.float64) - zq.astype(np.float64)) ** 2).sum(axis=1))
        assert np.all(s_lb <= true + 1e-3)
        qp = oracle.paa64(zq, 16)
        ref = np.array([oracle.mindist(qp, W[i], W[i], 256, 256) for i in range(0, case[0], 7)])
        np.testing.assert_allclose(s_lb[::7], ref, rtol=0, atol=2e-4)
        for l in range(0, len(lb) - 1, 5):
            members = perm[lb[l]:lb[l + 1]]
            assert l_lb[l] <= s_lb[members].min() + 1e-4


def test_stats_counters(msi):
    X = datagen.walks(11, 0, 8000, 256)
    ix = msi.msi_build(X, segments=16, leaf_capacity=64)
    msi.msi_query_stats_get(ix, reset=True)
    msi.msi_set_timing(ix, True)
    Q = datagen.paper_queries(8000, 256, count=6, data_seed=11)
    msi.msi_knn(ix, Q, 5)
    st = msi.msi_query_stats_get(ix)
    assert st["queries"] == 6
    assert st["leaves_total"] == 6 * ix.leaves
    assert 0 < st["series_refined"] <= 6 * 8000
    assert st["candidates"] >= 6 * 5 and st["rechecked"] >= 6 * 5
    # timed, the six queries run as one group of the batched chain: one series filter
    # and one row kernel launch timed for the group
    assert st["refine_launches"] == 1 and st["refine_ms"] > 0
    assert st["series_lower_bounded"] < 6 * 8000  # leaves were pruned
    # views, prep, seed, seed pick, leaf filter, front pick, front leaves, seed pick,
    # block filter, series filter, row refinement, finalize: once for the group
    assert st["kernel_launches"] == 12
    msi.msi_query_stats_get(ix, reset=True)
    msi.msi_knn(ix, Q[:1], 5)  # one query timed: its own chain
    st = msi.msi_query_stats_get(ix)
    assert st["refine_launches"] == 1 and st["kernel_launches"] == 10
    msi.msi_query_stats_get(ix, reset=True)
    msi.msi_set_timing(ix, False)
    # two queries in one call: the batched chain launches each stage once for both
    # (views, prep, seed, leaf filter, front pick, front leaves, block filter, series
    # filter, rows, finalize)
    msi.msi_knn(ix, Q[:2], 1)
    assert msi.msi_query_stats_get(ix)["kernel_launches"] == 10
    msi.msi_knn(ix, Q[:1], 40)  # one query, k > 32: its own chain, no register top-k
    assert msi.msi_query_stats_get(ix)["kernel_launches"] == 10 + 10
    msi.msi_schedule_set(ix, batch_chain=0)  # the query slots: a chain per query
    msi.msi_knn(ix, Q[:2], 1)
    assert msi.msi_query_stats_get(ix)["kernel_launches"] == 10 + 10 + 2 * 8


@pytest.mark.parametrize("chain", [1, 0])
def test_batched_slots_match_single_queries_and_oracle(msi, chain):
    """Queries run together (chain = 1: the batched chain, in groups of 4 queries per
    launch; chain = 0: concurrent query slots) give, for each query, the answer it gets
    alone, which is the oracle's; a query whose bounded lists overflow (many exact
    ties) is handed back to the full-capacity workspace."""
    n, length = 6000, 256
    X = datagen.walks(201, 0, n, length)
    X[1000:3500] = X[999]  # 2501 identical series: every one is a tie at distance 0
    Z = oracle.summarise(X, 16, 256)[0]
    Q = np.concatenate([datagen.paper_queries(n, length, count=7, data_seed=201), X[[999, 3000]]])
    for k in (1, 5, 32, 100):
        batched = msi.msi_build(X, segments=16, leaf_capacity=64, query_slots=3, slot_capacity=1024)
        msi.msi_schedule_set(batched, batch_chain=chain, batch_group=4, batch_share=2)
        single = msi.msi_build(X, segments=16, leaf_capacity=64, query_slots=1)
        ids_b, d_b = msi.msi_knn(batched, Q, k)
        for i, q in enumerate(Q):
            ids_s, d_s = msi.msi_knn(single, Q[i:i + 1], k)
            assert np.array_equal(ids_b[i], ids_s[0]) and np.array_equal(d_b[i], d_s[0])
            oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
            assert np.array_equal(ids_b[i], oid), (k, i)
        assert ids_b[-2][0] == 999 and list(ids_b[-1][:min(k, 3)]) == [999, 1000, 1001][:min(k, 3)]


@pytest.mark.parametrize("chain", [1, 0])
def test_repeated_batched_shape_replays_with_new_pointers(msi, chain):
    """A batched call shape (queries, k) seen before runs as a captured CUDA graph that
    takes its queries and outputs from a per-call descriptor: calls of the same shape
    with other query sets and other output buffers (host, device, with and without the
    FP64 distances) each give the oracle's answers, and every kernel is counted."""
    import torch
    n, length, nq, k = 6000, 256, 9, 5
    X = datagen.walks(211, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    sets = [datagen.paper_queries(n, length, count=nq, data_seed=211, fresh_seed=30 + j, pick_seed=40 + j)
            for j in range(3)]
    want = [[oracle.knn_scan(Z, oracle.znorm(q)[0], k)[0] for q in Q] for Q in sets]
    ix = msi.msi_build(X, segments=16, leaf_capacity=64, query_slots=4)
    msi.msi_schedule_set(ix, batch_chain=chain, batch_group=4)
    msi.msi_query_stats_get(ix, reset=True)
    calls = 0
    for rep in range(2):
        for j, Q in enumerate(sets):
            ids, d = msi.msi_knn(ix, Q, k)  # host buffers
            Qd = torch.from_numpy(Q).cuda()
            ids_d, d_d = msi.msi_knn(ix, Qd, k)  # fresh device buffers
            ids_x, d_x, d64_x = msi.msi_knn_ex(ix, Qd, k)
            calls += 3
            for i in range(nq):
                assert np.array_equal(ids[i], want[j][i]), (rep, j, i)
                assert np.array_equal(ids_d[i].cpu().numpy(), want[j][i]), (rep, j, i)
                assert np.array_equal(ids_x[i].cpu().numpy(), want[j][i]), (rep, j, i)
            assert np.array_equal(d, d_d.cpu().numpy()) and np.array_equal(d, d_x.cpu().numpy())
            assert np.all(d64_x.cpu().numpy() >= 0)
    st = msi.msi_query_stats_get(ix)
    assert st["queries"] == calls * nq
    # per call: 3 groups of at most 4 queries x 12 stages (k > 1), or 9 chains of 10
    assert st["kernel_launches"] == calls * (3 * 12 if chain else nq * 10)
    ix.close()


def test_autotune_keeps_answers_and_picks_a_measured_schedule(msi):
    """The batched-schedule autotuner times query slots x grid shares on the caller's
    queries and keeps the fastest; answers before and after are identical and the
    oracle's, and bad arguments are refused without changing the schedule."""
    import torch
    n, length, nq, k = 30000, 256, 24, 3
    X = datagen.walks(221, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    Q = datagen.paper_queries(n, length, count=nq, data_seed=221)
    ix = msi.msi_build(X, segments=16, leaf_capacity=200)
    before = msi.msi_knn(ix, Q, k)
    Qd = torch.from_numpy(Q).cuda()
    with pytest.raises(msi.MsiError):
        msi.msi_autotune(ix, Qd[:1], k)  # one query cannot be batched
    tr = msi.msi_autotune(ix, Qd, k, reps=2)
    if tr["batch_chain"]:
        assert tr["batch_group"] in (24, 128) and tr["batch_share"] in (1, 2, 4, 8)
    else:
        assert tr["query_slots"] in (4, 8, 12, 16, 24, 32)
        assert 1 <= tr["grid_share"] <= min(6, tr["query_slots"])
    # the index's own schedule, 4 batched-chain schedules, 2 with the tensor-core filter
    # and 29 slot schedules
    assert tr["candidates"] == 36 and tr["queries_per_s"] >= tr["default_queries_per_s"] > 0
    sched = msi.msi_schedule_get(ix)
    assert sched["batch_chain"] == tr["batch_chain"]
    after = msi.msi_knn(ix, Q, k)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    for i, q in enumerate(Q):
        oid, _ = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
        assert np.array_equal(after[0][i], oid), i
    ix.close()


@pytest.mark.parametrize("k,order", [(1, 0), (10, 0), (1, 1), (10, 1)])
def test_mixed_shapes_match_oracle(msi, k, order):
    """The harder value distributions (noisy sinusoids, Laplace-step walks with spike
    bursts), with the fresh-draw-plus-noise queries of that workload; order = 1 refines
    the survivors in ascending bound order (the same answers)."""
    n, length = 20000, 256
    X = datagen.mixed(4, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    Q = datagen.mixed_queries(count=12)
    ix = msi.msi_build(X, segments=16, cardinality=256, leaf_capacity=128)
    msi.msi_schedule_set(ix, batch_chain=1, batch_order=order)
    ids, d = msi.msi_knn(ix, Q, k)
    for i, q in enumerate(Q):
        oid, od2 = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
        assert np.array_equal(ids[i], oid), (k, i)
        np.testing.assert_allclose(d[i], np.sqrt(od2), rtol=RTOL, atol=1e-6)
