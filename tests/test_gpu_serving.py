"""The serving loop: requests for two resident indexes of different lengths, with
k from 1 to 100, submitted from two threads into a server with several slots per
index (continuous batching) and into a strictly one-at-a-time server. Each answer
must be the one the same query gets alone through msi_knn (and the oracle's), also
when a slot's bounded lists overflow and the query is rerun."""
import threading

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


def test_server_answers_equal_single_queries():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as msi

    XA = datagen.walks(301, 0, 20000, 256)
    XA[5000:6500] = XA[4999]  # 1501 ties: overflows the small slots below
    XB = datagen.mixed(302, 0, 8000, 128)
    A = msi.msi_build(XA, segments=16, leaf_capacity=64, query_slots=1)
    B = msi.msi_build(XB, segments=16, leaf_capacity=64, query_slots=1)
    rng = np.random.default_rng(3)
    reqs = []
    QA = np.concatenate([datagen.paper_queries(20000, 256, count=16, data_seed=301), XA[[4999, 5500]]])
    QB = datagen.mixed_queries(count=16, length=128, query_seed=303)
    for i, q in enumerate(QA):
        reqs.append((0, q, int(rng.choice([1, 5, 33, 100]))))
    for i, q in enumerate(QB):
        reqs.append((1, q, int(rng.choice([1, 7, 32, 64]))))
    order = rng.permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    want = [msi.msi_knn([A, B][ix], q[None, :], k) for ix, q, k in reqs]  # alone, before the servers

    for opts in (dict(slots_per_index=4, slot_capacity=1024), dict(slots_per_index=1, max_inflight=1)):
        srv = msi.Server([A, B], **opts)
        tickets = [None] * len(reqs)

        def submit(part):
            for j in part:
                ix, q, k = reqs[j]
                tickets[j] = srv.submit(ix, q, k)

        th = [threading.Thread(target=submit, args=(range(p, len(reqs), 2),)) for p in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for j, (ix, q, k) in enumerate(reqs):
            ids, d, ms = srv.wait(tickets[j], k)
            assert np.array_equal(ids, want[j][0][0]), (opts, j)
            assert np.array_equal(d, want[j][1][0]), (opts, j)
            assert ms >= 0.0
        st = srv.stats()
        assert st["completed"] == len(reqs)
        if opts.get("slot_capacity"):
            assert st["reruns"] >= 1  # the tie-heavy queries went back to the full workspace
        srv.close()

    ZA = oracle.summarise(XA, 16, 256)[0]
    for j, (ix, q, k) in enumerate(reqs[:10]):
        X = XA if ix == 0 else XB
        Z = ZA if ix == 0 else oracle.summarise(XB, 16, 256)[0]
        oid, _ = oracle.knn_scan(Z, oracle.znorm(q)[0], k)
        assert np.array_equal(want[j][0][0], oid)
