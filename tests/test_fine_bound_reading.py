"""The fine PAA bound as read from Section II-B (the PAA lower bound, over finer
segments than the iSAX word) with the fp16 storage margin the kernels subtract: on
plain CPU arithmetic it never exceeds the squared Euclidean distance, nor the squared
DTW distance when the query side is the window-widened envelope. This pins the
reading, not the GPU code (the GPU tests compare that with the oracle's answers)."""
import numpy as np

import datagen
import oracle


def fine_means_fp16(Z, wf):
    """Segment means of the fp32 z values, rounded to the nearest fp16."""
    n, length = Z.shape
    return Z.astype(np.float64).reshape(n, wf, length // wf).mean(-1).astype(np.float32).astype(np.float16)


def fine_lb2(h16, up, lo, sf):
    """sf * sum_j gap_j^2, each gap taken half an fp16 ulp (plus 2^-25) short."""
    h = h16.astype(np.float64)
    e = np.abs(h) * 2.0 ** -11 + 2.0 ** -25
    g = np.maximum(0.0, np.maximum(h - up - e, lo - h - e))
    return sf * (g * g).sum(-1)


def test_fine_bound_never_exceeds_the_euclidean_distance():
    n, length, wf = 3000, 256, 64
    X = datagen.walks(41, 0, n, length)
    Z = oracle.summarise(X, 16, 256)[0]
    H = fine_means_fp16(Z, wf)
    # with exact members among the queries: distance 0, where only the margin keeps the
    # fp16-rounded means from bounding above it
    Q = np.concatenate([datagen.paper_queries(n, length, count=16, data_seed=41), X[[5, 777]]])
    tighter = 0
    for q in Q:
        zq = oracle.znorm(q)[0].astype(np.float64)
        qm = zq.reshape(wf, length // wf).mean(-1)
        d2 = ((Z.astype(np.float64) - zq) ** 2).sum(-1)
        lb = fine_lb2(H, qm, qm, length // wf)
        assert np.all(lb <= d2 * (1 + 1e-6) + 1e-9), float((lb - d2).max())
        # finer segments bound more tightly than the 16-segment PAA on these series
        q16 = zq.reshape(16, 16).mean(-1)
        lb16 = 16 * ((Z.astype(np.float64).reshape(n, 16, 16).mean(-1) - q16) ** 2).sum(-1)
        tighter += int(np.median(lb / np.maximum(lb16, 1e-12)) > 1.0)
    assert tighter == len(Q)
    assert fine_lb2(H[5], Z[5].astype(np.float64).reshape(wf, -1).mean(-1),
                    Z[5].astype(np.float64).reshape(wf, -1).mean(-1), length // wf) == 0.0


def test_fine_bound_never_exceeds_dtw_with_the_window_envelope():
    n, length, r = 300, 64, 6
    wf = 64  # one point per segment: the bound becomes LB_Keogh with the fp16 margin
    X = datagen.walks(42, 0, n, length)
    Z = oracle.summarise(X, 8, 256)[0]
    H = fine_means_fp16(Z, wf)
    Q = np.concatenate([datagen.paper_queries(n, length, count=4, data_seed=42), X[[7]]])
    for q in Q:
        zq = oracle.znorm(q)[0].astype(np.float64)
        up = np.array([zq[max(0, t - r):t + r + 1].max() for t in range(length)])
        lo = np.array([zq[max(0, t - r):t + r + 1].min() for t in range(length)])
        ids, d2 = oracle.knn_scan_dtw(Z, zq.astype(np.float32), n, r)
        dtw2 = np.empty(n)
        dtw2[ids] = d2
        lb = fine_lb2(H, up, lo, 1)
        assert np.all(lb <= dtw2 * (1 + 1e-6) + 1e-9), float((lb - dtw2).max())
    # with 4-point segments the envelope is reduced per segment (max of U, min of L)
    wf4 = 16
    H4 = fine_means_fp16(Z, wf4)
    for q in Q:
        zq = oracle.znorm(q)[0].astype(np.float64)
        up = np.array([zq[max(0, j * 4 - r):min(length, j * 4 + 4 + r)].max() for j in range(wf4)])
        lo = np.array([zq[max(0, j * 4 - r):min(length, j * 4 + 4 + r)].min() for j in range(wf4)])
        ids, d2 = oracle.knn_scan_dtw(Z, zq.astype(np.float32), n, r)
        dtw2 = np.empty(n)
        dtw2[ids] = d2
        assert np.all(fine_lb2(H4, up, lo, 4) <= dtw2 * (1 + 1e-6) + 1e-9)
