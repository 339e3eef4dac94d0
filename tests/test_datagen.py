"""The seeded input generators: Philox known answers, elementary-function accuracy,
distribution moments, the random-walk recipe and slice reproducibility. CPU only."""
import os

import numpy as np
import pytest

import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert list(datagen.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


def test_ln_and_sincos_accuracy():
    xs = np.concatenate([np.geomspace(2.0 ** -24, 1.0, 3000), [1.0, 0.5, 0.75]]).astype(np.float32)
    for x in xs:
        assert abs(datagen.ln(x) - np.log(np.float64(x))) <= 4e-7 * max(1.0, abs(np.log(np.float64(x))))
    for u in np.linspace(0, 1, 4001, endpoint=False).astype(np.float32):
        s, c = datagen.sincos_2pi(u)
        assert abs(s - np.sin(2 * np.pi * np.float64(u))) < 1e-6
        assert abs(c - np.cos(2 * np.pi * np.float64(u))) < 1e-6


def test_normal_moments():
    z = datagen.normals(5, 0, 0, 1_000_000).astype(np.float64)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1) < 5e-3
    assert abs((z ** 3).mean()) < 2e-2
    assert abs((z ** 4).mean() - 3) < 5e-2


def test_random_walk_recipe_and_slices():
    w = datagen.walks(9, 0, 6, 64)
    for i in range(6):
        e = datagen.normals(9, 0, i, 64)
        want = np.empty(64, np.float32)
        acc = np.float32(0)
        for t in range(64):
            acc = e[t] if t == 0 else np.float32(acc + e[t])
            want[t] = acc
        assert np.array_equal(w[i], want)
    assert np.array_equal(datagen.walks(9, 2, 3, 64), w[2:5])
    assert not np.array_equal(datagen.walks(10, 0, 1, 64)[0], w[0])


def test_noisy_copies_and_picks():
    ids = datagen.pick(2, 0, 1000, 12345)
    assert ids.min() >= 0 and ids.max() < 12345 and len(np.unique(ids)) > 900
    q = datagen.noisy_copies(0, 2, ids[:3], np.float32([0.0, 0.1, 1.0]), 128)
    base = datagen.walks(0, 0, 12345, 128)[ids[:3]]
    assert np.array_equal(q[0], base[0])
    assert 0.05 < np.std(q[1] - base[1]) < 0.2
    assert 0.5 < np.std(q[2] - base[2]) < 2.0
    qs = datagen.paper_queries(12345, 128, count=100)
    assert qs.shape == (100, 128) and qs.dtype == np.float32


def test_mixed_shapes():
    X = datagen.mixed(4, 0, 4000, 256)
    assert np.isfinite(X).all()
    sd = X.std(axis=1)
    sinus = sd < 2.0  # sinusoid + N(0, 0.3): std about sqrt(0.5 + 0.3)
    assert 0.4 < sinus.mean() < 0.6
    assert np.all(np.abs(sd[sinus] - np.sqrt(0.8)) < 0.25)
    walks = X[~sinus]
    steps = np.abs(np.diff(walks, axis=1))
    # one burst of 13 steps x10 per walk: the largest steps sit in one run
    big = steps > 8.0
    assert big.any(axis=1).mean() > 0.5
    assert np.array_equal(datagen.mixed(4, 100, 5, 256), X[100:105])
    Q = datagen.mixed_queries(count=5)
    assert Q.shape == (5, 256) and 0.2 < np.std(Q - datagen.mixed(5, 0, 5, 256)) < 0.45
