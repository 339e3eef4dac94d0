"""CPU oracle for exact k-NN over iSAX-summarised data series.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
benchmark's CPU-baseline leg, never by the product package. It shares no code with
the CUDA library. See oracle.c for the arithmetic and the passages each function
follows.

Parity status of each function (what pins it, tests/test_oracle_pins.py):
  breakpoints / thresholds   pinned (textbook quantiles, symmetry, library ppf)
  znorm                      pinned (FP64 library moments, invariants, constant case)
  paa                        pinned (closed forms, FP64 mean)
  sax                        pinned (monotonicity, prefix property, equiprobability)
  mindist                    pinned (lower-bound property by brute force, special cases)
  knn_scan                   pinned (brute force, self-match, duplicates, k = N)
  knn_index                  pinned (equals knn_scan)
  dtw_sq                     pinned (brute force over warping paths, r = 0 is the
                             squared Euclidean distance, hand-worked cases)
  envelope / lb_keogh        pinned (closed form on monotone series, bound property)
  mindist_env                pinned (bounds LB_Keogh by brute force, reduces to the
                             PAA mindist for segment-constant queries at r = 0)
  knn_scan_dtw / knn_index_dtw  pinned (brute force, self-match, index equals scan)
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.orc_breakpoints.argtypes = [i32, vp]
        L.orc_thresholds.argtypes = [i32, vp]
        L.orc_znorm.argtypes = [vp, i32, vp, vp, vp]
        L.orc_znorm.restype = i32
        L.orc_paa.argtypes = [vp, i32, i32, vp]
        L.orc_sax.argtypes = [vp, i32, i32, vp, vp]
        L.orc_summarise.argtypes = [vp, i64, i32, i32, i32, vp, vp, vp, vp]
        L.orc_summarise.restype = i64
        L.orc_mindist.argtypes = [vp, vp, vp, i32, i32, i32, vp]
        L.orc_mindist.restype = f64
        L.orc_paa64.argtypes = [vp, i32, i32, vp]
        L.orc_sqdist.argtypes = [vp, vp, i32]
        L.orc_sqdist.restype = f64
        L.orc_knn_scan.argtypes = [vp, i64, i32, vp, i32, vp, vp]
        L.orc_knn_index.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, i32, f64, vp, vp]
        L.orc_knn_index.restype = i64
        L.orc_dtw_sq.argtypes = [vp, vp, i32, i32]
        L.orc_dtw_sq.restype = f64
        L.orc_envelope.argtypes = [vp, i32, i32, vp, vp]
        L.orc_lb_keogh.argtypes = [vp, vp, vp, i32]
        L.orc_lb_keogh.restype = f64
        L.orc_paa_envelope.argtypes = [vp, vp, i32, i32, vp, vp]
        L.orc_mindist_env.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp]
        L.orc_mindist_env.restype = f64
        L.orc_knn_scan_dtw.argtypes = [vp, i64, i32, vp, i32, i32, vp, vp]
        L.orc_knn_index_dtw.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, i32, i32, f64, vp, vp]
        L.orc_knn_index_dtw.restype = i64
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def breakpoints(c):
    """beta_i = Phi^-1(i/c), i = 1..c-1 (float64)."""
    out = np.empty(c - 1, dtype=np.float64)
    lib().orc_breakpoints(c, _p(out))
    return out


def thresholds(c):
    """Smallest float32 >= beta_i, i = 1..c-1."""
    out = np.empty(c - 1, dtype=np.float32)
    lib().orc_thresholds(c, _p(out))
    return out


def znorm(x):
    """Canonical fp32 z-normalisation of one series -> (z, flag, mu, 1/sigma);
    flag 0 normal, 1 constant (z = 0), -1 non-finite."""
    x = _f32(x)
    z = np.empty_like(x)
    mu, r = ctypes.c_float(), ctypes.c_float()
    flag = lib().orc_znorm(_p(x), len(x), _p(z), ctypes.byref(mu), ctypes.byref(r))
    return z, flag, mu.value, r.value


def paa(z, w):
    z = _f32(z)
    out = np.empty(w, dtype=np.float32)
    lib().orc_paa(_p(z), len(z), w, _p(out))
    return out


def sax(paa_values, c):
    p = _f32(paa_values)
    t = thresholds(c)
    out = np.empty(len(p), dtype=np.uint8)
    lib().orc_sax(_p(p), len(p), c, _p(t), _p(out))
    return out


def summarise(X, w, c, want_z=True, want_paa=True):
    """Row-wise z-norm + PAA + SAX of X [N, n] -> (Z, PAA, words, flags)."""
    X = _f32(X)
    N, n = X.shape
    Z = np.empty_like(X) if want_z else None
    P = np.empty((N, w), dtype=np.float32) if want_paa else None
    W = np.empty((N, w), dtype=np.uint8)
    F = np.empty(N, dtype=np.int32)
    lib().orc_summarise(_p(X), N, n, w, c, _p(Z), _p(P), _p(W), _p(F))
    return Z, P, W, F


def paa64(z, w):
    z = _f32(z)
    out = np.empty(w, dtype=np.float64)
    lib().orc_paa64(_p(z), len(z), w, _p(out))
    return out


def mindist(qpaa64, lo, hi, n, c):
    """iSAX lower bound between a query (FP64 PAA) and symbol ranges [lo, hi]."""
    q = np.ascontiguousarray(qpaa64, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.uint8)
    hi = np.ascontiguousarray(hi, dtype=np.uint8)
    beta = breakpoints(c)
    return lib().orc_mindist(_p(q), _p(lo), _p(hi), len(q), n, c, _p(beta))


def sqdist(a, b):
    a, b = _f32(a), _f32(b)
    return lib().orc_sqdist(_p(a), _p(b), len(a))


def knn_scan(Z, zq, k):
    """Exact k-NN by FP64 serial scan: (ids int64[k], d2 float64[k]), ties -> lower id."""
    Z = _f32(Z)
    zq = _f32(zq)
    ids = np.empty(k, dtype=np.int64)
    d2 = np.empty(k, dtype=np.float64)
    lib().orc_knn_scan(_p(Z), Z.shape[0], Z.shape[1], _p(zq), k, _p(ids), _p(d2))
    return ids, d2


def knn_index(Z, words, zq, k, c=256, cap=2000, slack=1e-4):
    """Exact k-NN through the oracle's own flat index: (ids, d2, real_distance_count)."""
    Z = _f32(Z)
    W = np.ascontiguousarray(words, dtype=np.uint8)
    zq = _f32(zq)
    ids = np.empty(k, dtype=np.int64)
    d2 = np.empty(k, dtype=np.float64)
    real = lib().orc_knn_index(_p(Z), _p(W), Z.shape[0], Z.shape[1], W.shape[1], c, cap, _p(zq), k,
                               slack, _p(ids), _p(d2))
    return ids, d2, real


# ------------------------------------------------------------------ DTW
def dtw_sq(a, b, r):
    """FP64 squared DTW of two fp32 series with a Sakoe-Chiba band of half-width r."""
    a, b = _f32(a), _f32(b)
    return lib().orc_dtw_sq(_p(a), _p(b), len(a), r)


def envelope(q, r):
    """LB_Keogh envelope (U, L) of a series for warping window r (float32)."""
    q = _f32(q)
    U, L = np.empty_like(q), np.empty_like(q)
    lib().orc_envelope(_p(q), len(q), r, _p(U), _p(L))
    return U, L


def lb_keogh(U, L, b):
    """Squared LB_Keogh of series b against the envelope (U, L), FP64."""
    U, L, b = _f32(U), _f32(L), _f32(b)
    return lib().orc_lb_keogh(_p(U), _p(L), _p(b), len(b))


def paa_envelope(U, L, w):
    """Per-segment max of U and min of L (FP64)."""
    U, L = _f32(U), _f32(L)
    Uh, Lh = np.empty(w), np.empty(w)
    lib().orc_paa_envelope(_p(U), _p(L), len(U), w, _p(Uh), _p(Lh))
    return Uh, Lh


def mindist_env(Uh, Lh, lo, hi, n, c):
    """DTW lower bound between a query's PAA envelope and symbol ranges [lo, hi]."""
    Uh = np.ascontiguousarray(Uh, dtype=np.float64)
    Lh = np.ascontiguousarray(Lh, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.uint8)
    hi = np.ascontiguousarray(hi, dtype=np.uint8)
    beta = breakpoints(c)
    return lib().orc_mindist_env(_p(Uh), _p(Lh), _p(lo), _p(hi), len(Uh), n, c, _p(beta))


def knn_scan_dtw(Z, zq, k, r):
    """Exact k-NN under DTW (window r) by FP64 serial scan: (ids, DTW^2), ties -> lower id."""
    Z = _f32(Z)
    zq = _f32(zq)
    ids = np.empty(k, dtype=np.int64)
    d2 = np.empty(k, dtype=np.float64)
    lib().orc_knn_scan_dtw(_p(Z), Z.shape[0], Z.shape[1], _p(zq), k, r, _p(ids), _p(d2))
    return ids, d2


def knn_index_dtw(Z, words, zq, k, r, c=256, cap=2000, slack=1e-4):
    """Exact k-NN under DTW through the oracle's flat index: (ids, DTW^2, real_distance_count)."""
    Z = _f32(Z)
    W = np.ascontiguousarray(words, dtype=np.uint8)
    zq = _f32(zq)
    ids = np.empty(k, dtype=np.int64)
    d2 = np.empty(k, dtype=np.float64)
    real = lib().orc_knn_index_dtw(_p(Z), _p(W), Z.shape[0], Z.shape[1], W.shape[1], c, cap, _p(zq), k, r,
                                   slack, _p(ids), _p(d2))
    return ids, d2, real
