"""Pins of the CPU oracle to facts fixed outside it: textbook quantiles, library
routines, closed forms, invariants and brute force on tiny inputs. CPU only.

Each group is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, an off-by-one symbol) fails a test.
"""
import os

import numpy as np
import pytest
from scipy.stats import norm, chisquare

import datagen
import oracle

U32 = np.float32(2.0) ** -24  # unit roundoff of fp32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _z64(x):
    x = np.asarray(x, dtype=np.float64)
    return (x - x.mean()) / x.std()


# ------------------------------------------------------------------ breakpoints
def test_breakpoints_match_golden_quantiles():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "normal_quantiles.txt")) if l.strip() and l[0] != "#"]
    for c in (4, 8):
        b = oracle.breakpoints(c)
        want = [float(r[3]) for r in rows if int(r[0]) == c]
        assert len(b) == c - 1
        np.testing.assert_allclose(b, want, rtol=0, atol=2e-15)


@pytest.mark.parametrize("c", [2, 4, 16, 64, 256])
def test_breakpoints_library_symmetry_equiprobable(c):
    b = oracle.breakpoints(c)
    np.testing.assert_allclose(b, norm.ppf(np.arange(1, c) / c), rtol=0, atol=1e-13)
    np.testing.assert_allclose(b, -b[::-1], rtol=0, atol=1e-15)
    assert np.all(np.diff(b) > 0)
    probs = np.diff(np.concatenate([[0.0], norm.cdf(b), [1.0]]))
    np.testing.assert_allclose(probs, 1.0 / c, rtol=0, atol=1e-12)


def test_thresholds_are_smallest_float_at_or_above_breakpoint():
    b = oracle.breakpoints(256)
    t = oracle.thresholds(256)
    assert t[127] == 0.0 and b[127] == 0.0
    assert np.all(t.astype(np.float64) >= b)
    below = np.nextafter(t, np.float32(-np.inf)).astype(np.float64)
    assert np.all(below < b)


# ------------------------------------------------------------- z-normalisation
def test_znorm_matches_fp64_definition_and_invariants():
    X = datagen.walks(7, 0, 200, 256)
    for x in X:
        z, flag, mu, r = oracle.znorm(x)
        assert flag == 0
        x64 = x.astype(np.float64)
        ratio = 1.0 + abs(x64.mean()) / x64.std()
        # fp32 two-pass moments: a few ulps, scaled by the mean/std ratio
        assert np.max(np.abs(z - _z64(x))) <= 64 * U32 * ratio * 4
        assert abs(z.astype(np.float64).mean()) <= 16 * U32 * ratio
        assert abs(z.astype(np.float64).var() - 1.0) <= 64 * U32


def test_znorm_constant_and_nonfinite():
    z, flag, _, _ = oracle.znorm(np.full(256, 3.25, np.float32))
    assert flag == 1 and np.all(z == 0)
    z, flag, _, _ = oracle.znorm(np.full(64, 0.1, np.float32))
    assert flag == 1 and np.all(z == 0)
    x = np.full(128, 1000.0, np.float32)
    x[5] += np.float32(1e-4)  # relative spread far below fp32 resolution of the mean
    assert oracle.znorm(x)[1] == 1
    x = datagen.walks(1, 0, 1, 256)[0]
    x[17] = np.nan
    assert oracle.znorm(x)[1] == -1
    x[17] = np.inf
    assert oracle.znorm(x)[1] == -1


def test_znorm_affine_invariance():
    x = datagen.walks(3, 5, 1, 256)[0]
    z = oracle.znorm(x)[0]
    z2 = oracle.znorm(np.float32(3.5) * x + np.float32(-20.0))[0]
    z3 = oracle.znorm(np.float32(-2.0) * x)[0]
    assert np.max(np.abs(z - z2)) < 2e-5
    assert np.max(np.abs(z + z3)) < 2e-5


# ------------------------------------------------------------------------ PAA
def test_paa_piecewise_constant_and_ramp_closed_forms():
    w, n = 16, 256
    vals = np.linspace(-2, 2, w).astype(np.float32)
    assert np.array_equal(oracle.paa(np.repeat(vals, n // w), w), vals)
    ramp = np.arange(n, dtype=np.float32)
    s = n // w
    assert np.array_equal(oracle.paa(ramp, w), (np.arange(w) * s + (s - 1) / 2).astype(np.float32))
    # 8 segments of a length-128 series, 4 segments of 64 points
    assert np.array_equal(oracle.paa(np.arange(128, dtype=np.float32), 8), (np.arange(8) * 16 + 7.5).astype(np.float32))


@pytest.mark.parametrize("n,w", [(256, 16), (128, 16), (1024, 16), (96, 16), (60, 4), (256, 8)])
def test_paa_is_segment_mean(n, w):
    X = datagen.walks(11, 0, 20, n)
    for x in X:
        z = oracle.znorm(x)[0]
        want = z.astype(np.float64).reshape(w, n // w).mean(axis=1)
        got = oracle.paa(z, w)
        scale = np.abs(z).reshape(w, n // w).mean(axis=1) + 1e-30
        assert np.all(np.abs(got - want) <= 8 * U32 * np.log2(n) * scale + 1e-12)


# ------------------------------------------------------------------------ SAX
def test_sax_small_table_by_hand():
    # cardinality 4: regions (-inf,-0.674), [-0.674,0), [0,0.674), [0.674,inf)
    assert list(oracle.sax([-1.0, -0.5, 0.0, 0.7, 0.674, -0.6745], 4)) == [0, 1, 2, 3, 2, 0]


def test_sax_monotone_and_boundaries():
    grid = np.linspace(-4, 4, 200001).astype(np.float32)
    syms = oracle.sax(grid, 256).astype(int)
    assert np.all(np.diff(syms) >= 0)
    assert syms[0] == 0 and syms[-1] == 255 and len(np.unique(syms)) == 256
    t = oracle.thresholds(256)
    assert list(oracle.sax(t, 256).astype(int)) == list(range(1, 256))
    below = np.nextafter(t, np.float32(-np.inf))
    assert list(oracle.sax(below, 256).astype(int)) == list(range(0, 255))


def test_sax_prefix_property():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(20000).astype(np.float32) * 1.3
    s256 = oracle.sax(p, 256).astype(int)
    for b in range(1, 8):
        assert np.array_equal(s256 >> (8 - b), oracle.sax(p, 2 ** b).astype(int))


def test_sax_equiprobable_regions():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(1_000_000).astype(np.float32)
    counts = np.bincount(oracle.sax(p, 256), minlength=256)
    assert chisquare(counts).pvalue > 1e-4


# -------------------------------------------------------------------- mindist
def test_mindist_hand_example():
    q = np.array([-1.0, 1.0])
    # symbol 3 of 4 covers [0.6745, inf), symbol 0 covers (-inf, -0.6745); s = 2
    lb = oracle.mindist(q, [3, 0], [3, 0], n=4, c=4)
    gap = 1.0 + 0.6744897501960817
    assert abs(lb - np.sqrt(2 * 2 * gap * gap)) < 1e-12
    assert oracle.mindist(q, [0, 0], [3, 3], n=4, c=4) == 0.0
    # symbol 2 covers [0, 0.6745): gaps 1 (below) and 1 - 0.6745 (above)
    want = np.sqrt(2 * (1.0 + (1.0 - 0.6744897501960817) ** 2))
    assert abs(oracle.mindist(q, [2, 2], [2, 2], n=4, c=4) - want) < 1e-12


@pytest.mark.parametrize("n,w", [(16, 4), (32, 16), (64, 16), (256, 16)])
def test_mindist_lower_bounds_true_distance_brute_force(n, w):
    X = datagen.walks(21, 0, 400, n)
    Z, _, W, _ = oracle.summarise(X, w, 256)
    Q = datagen.walks(22, 0, 5, n)
    for q in Q:
        zq = oracle.znorm(q)[0]
        qp = oracle.paa64(zq, w)
        d = np.sqrt(((Z.astype(np.float64) - zq.astype(np.float64)) ** 2).sum(axis=1))
        lb = np.array([oracle.mindist(qp, W[i], W[i], n, 256) for i in range(len(Z))])
        assert np.all(lb <= d + 1e-5)
        assert np.mean(lb > 0) > 0.5  # the bound is not trivially zero
        lo, hi = W.min(axis=0), W.max(axis=0)
        env = oracle.mindist(qp, lo, hi, n, 256)
        assert env <= lb.min() + 1e-12
        own = oracle.sax(oracle.paa(zq, w), 256)
        assert oracle.mindist(qp, np.minimum(own, lo), np.maximum(own, hi), n, 256) == 0.0


def test_mindist_of_nested_envelopes_is_monotone():
    # The block filter bounds a block of 32 positions by the envelope of its halves
    # of 16 (and could go down to quarters of 8): a symbol range that contains another
    # bounds no higher, so every word's bound is at least its quarter's, which is at
    # least its half's, which is at least its block's; and the finer envelopes do prune
    # more (some half bound strictly exceeds its block's).
    n, w = 64, 16
    X = datagen.walks(23, 0, 512, n)
    Z, _, W, _ = oracle.summarise(X, w, 256)
    q = oracle.znorm(datagen.walks(24, 0, 1, n)[0])[0]
    qp = oracle.paa64(q, w)
    d = np.sqrt(((Z.astype(np.float64) - q.astype(np.float64)) ** 2).sum(axis=1))

    def bounds(width):
        g = W.reshape(-1, width, w)
        return np.array([oracle.mindist(qp, b.min(axis=0), b.max(axis=0), n, 256) for b in g])

    b32, b16, b8, b1 = bounds(32), bounds(16), bounds(8), bounds(1)
    assert np.all(b32 <= b16.reshape(-1, 2).min(axis=1) + 1e-12)
    assert np.all(b16 <= b8.reshape(-1, 2).min(axis=1) + 1e-12)
    assert np.all(b8 <= b1.reshape(-1, 8).min(axis=1) + 1e-12)
    assert np.all(b1 <= d + 1e-5)
    assert np.any(b16.reshape(-1, 2).max(axis=1) > b32 + 1e-9)


def test_mindist_equals_paa_distance_in_the_limit_of_fine_regions():
    # With the query's own symbols, each gap is at most the width of a region,
    # so LB(q, word(q)) == 0; a word whose every segment lies far away gives the
    # closed-form gap to the nearest breakpoint.
    q = np.zeros(16)
    lb = oracle.mindist(q, np.full(16, 255), np.full(16, 255), n=256, c=256)
    assert abs(lb - np.sqrt(16 * 16 * oracle.breakpoints(256)[-1] ** 2)) < 1e-12


# ---------------------------------------------------------------- exact k-NN
def _brute(Z, zq, k):
    d2 = ((Z.astype(np.float64) - zq.astype(np.float64)) ** 2).sum(axis=1)
    order = np.lexsort((np.arange(len(d2)), d2))[:k]
    return order, d2[order]


def test_knn_scan_brute_force():
    X = datagen.walks(31, 0, 3000, 256)
    Z = oracle.summarise(X, 16, 256)[0]
    for q in datagen.walks(32, 0, 4, 256):
        zq = oracle.znorm(q)[0]
        for k in (1, 5, 37):
            ids, d2 = oracle.knn_scan(Z, zq, k)
            bi, bd = _brute(Z, zq, k)
            assert np.array_equal(ids, bi)
            np.testing.assert_allclose(d2, bd, rtol=1e-12)


def test_sqdist_within_the_error_bound_of_the_exact_sum():
    """The FP64 distance against exact rational arithmetic (Section II-A's sum of
    squared differences of the fp32 values): a sequential FP64 sum of n rounded terms
    is within n 2^-53 of the exact value, relative; a dropped, doubled or mis-signed
    term is not."""
    from fractions import Fraction
    X = datagen.walks(33, 0, 6, 256)
    Z = oracle.summarise(X, 16, 256)[0]
    for a in range(3):
        for b in range(3, 6):
            exact = sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(Z[a], Z[b]))
            got = oracle.sqdist(Z[a], Z[b])
            assert abs(Fraction(got) - exact) <= exact * Fraction(256 + 2, 2 ** 53)
    assert oracle.sqdist(Z[0], Z[0]) == 0.0


def test_knn_scan_special_cases():
    X = datagen.walks(41, 0, 500, 128)
    Z = oracle.summarise(X, 16, 256)[0]
    ids, d2 = oracle.knn_scan(Z, Z[123], 1)
    assert ids[0] == 123 and d2[0] == 0.0
    Zd = Z.copy()
    Zd[400] = Zd[77]  # duplicate: lower id first
    ids, d2 = oracle.knn_scan(Zd, Zd[77], 2)
    assert list(ids) == [77, 400] and d2[1] == 0.0
    ids, d2 = oracle.knn_scan(Z, Z[0], len(Z))  # k = N: full order
    bi, bd = _brute(Z, Z[0], len(Z))
    assert np.array_equal(ids, bi)
    assert np.all(np.diff(d2) >= 0)


@pytest.mark.parametrize("k", [1, 10, 100])
def test_knn_index_equals_scan(k):
    X = datagen.walks(51, 0, 6000, 256)
    Z, _, W, _ = oracle.summarise(X, 16, 256)
    Q = datagen.paper_queries(6000, 256, count=8, data_seed=51, fresh_seed=52, pick_seed=53)
    for q in Q:
        zq = oracle.znorm(q)[0]
        ids, d2 = oracle.knn_scan(Z, zq, k)
        ids2, d22, real = oracle.knn_index(Z, W, zq, k, cap=64)
        assert np.array_equal(ids, ids2)
        assert np.array_equal(d2, d22)
        assert real < len(Z)  # the lower bounds pruned something
