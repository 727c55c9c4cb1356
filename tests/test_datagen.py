"""The seeded input generator (datagen/) against published vectors and its
defining properties.  CPU only."""
import math
import os

import numpy as np
import pytest

import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert datagen.philox4x32_10(ctr, key) == out


def test_ln_matches_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.random(2000), [2.0**-53, 1.0 - 2.0**-53, 1.0, 0.5, 0.70710678]])
    xs = xs[xs > 0]
    for x in xs:
        ref = math.log(x)
        got = datagen.ln(x)
        assert abs(got - ref) <= 4 * math.ulp(ref) + 1e-300, (x, got, ref)


def test_sincos_matches_libm():
    rng = np.random.default_rng(1)
    us = np.concatenate([rng.random(2000), np.arange(16) / 16.0])
    for u in us:
        s, c = datagen.sincos_turns(u)
        assert abs(s - math.sin(2 * math.pi * u)) < 1e-15
        assert abs(c - math.cos(2 * math.pi * u)) < 1e-15


def test_normals_are_standard():
    from scipy import stats
    z = np.array([datagen.normal_pair(7, r, d) for r in range(200) for d in range(100)]).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3


@pytest.mark.parametrize("kind", ["walk", "sine"])
def test_rows_are_independent_of_batching(kind):
    a = datagen.rows(kind, 3, 0, 20, 128)
    b = datagen.rows(kind, 3, 7, 5, 128, nthreads=1)
    np.testing.assert_array_equal(a[7:12], b)
    c = datagen.rows_at(kind, 3, [19, 2], 128)
    np.testing.assert_array_equal(c, a[[19, 2]])


@pytest.mark.parametrize("kind", ["walk", "sine"])
def test_rows_are_z_normalised(kind):
    X = datagen.rows(kind, 0, 0, 200, 256).astype(np.float64)
    assert np.abs(X.mean(axis=1)).max() < 1e-6
    assert np.abs(X.std(axis=1) - 1).max() < 1e-6


def test_random_walk_is_cumsum_of_the_normals():
    n = 64
    z = np.array([datagen.normal_pair(5, 11, d) for d in range(n // 2)]).ravel()
    x = np.cumsum(z)
    ref = ((x - x.mean()) / x.std()).astype(np.float32)
    got = datagen.rows("walk", 5, 11, 1, n)[0]
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-6)


def test_noisy_members_and_picks():
    N, n = 1000, 128
    Q, src = datagen.queries("walk", 0, N, n, 1, 5, 5, 0.01)
    assert Q.shape == (10, n) and Q.dtype == np.float32
    assert (src[:5] == -1).all() and ((src[5:] >= 0) & (src[5:] < N)).all()
    members = datagen.rows_at("walk", 0, src[5:], n)
    d = np.sqrt(((Q[5:].astype(np.float64) - members) ** 2).sum(axis=1))
    assert (d < 0.01 * math.sqrt(n) * 3).all()
    picks = datagen.pick_members(9, 0, 20000, 10)
    counts = np.bincount(picks, minlength=10)
    assert counts.min() > 1700 and counts.max() < 2300
