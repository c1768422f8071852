"""Pins of the oracle's detector-noise stage (Sec. 2.2: photon noise, dark current, RON,
pixel response non-uniformity, cross-talk added to the final frame).

The generator is pinned to its published known-answer vectors; the samplers to the
distributions they must produce (chi-square and Kolmogorov-Smirnov tests at fixed seeds,
thresholds far in the tails); the frame stage to closed forms with the random parts off.
"""
import json
import os

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["counter"]]
        key = [int(x, 16) for x in v["key"]]
        assert oracle.philox4x32_10(ctr, key) == [int(x, 16) for x in v["out"]]


def test_normal_pairs_are_standard_normal_and_uncorrelated():
    n = 20000
    z = np.array([oracle.normal_pair(77, q, 3, 1) for q in range(n)])
    for col in (0, 1):
        assert stats.kstest(z[:, col], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 4.0 / np.sqrt(n)
    # a different stream or detector gives a different sequence
    assert oracle.normal_pair(77, 5, 3, 1) != oracle.normal_pair(77, 5, 3, 0)
    assert oracle.normal_pair(77, 5, 3, 1) != oracle.normal_pair(77, 5, 4, 1)


@pytest.mark.parametrize("lam", [0.3, 2.5, 9.99, 10.0, 37.5, 1000.0, 40000.0])
def test_poisson_sampler_matches_the_distribution(lam):
    n = 20000
    k = np.array([oracle.poisson(lam, 1234, q, 0, q & 1) for q in range(n)])
    assert k.min() >= 0
    # chi-square over bins holding >= 20 expected counts (tails pooled)
    lo, hi = stats.poisson.ppf(1e-4, lam), stats.poisson.ppf(1 - 1e-4, lam)
    edges = np.unique(np.linspace(lo, hi + 1, 40).astype(int))
    cdf = stats.poisson.cdf(edges - 1, lam)
    probs = np.diff(np.concatenate([[0.0], cdf[1:], [1.0]]))
    counts = np.histogram(k, bins=np.concatenate([[-0.5], edges[1:] - 0.5, [np.inf]]))[0]
    keep = probs * n >= 20
    exp = probs[keep] * n
    obs = counts[keep].astype(float)
    exp *= obs.sum() / exp.sum()
    assert stats.chisquare(obs, exp).pvalue > 1e-4
    assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
    assert abs(k.var() / lam - 1) < 5 * np.sqrt(2.0 / n)


def test_poisson_of_zero_and_negative_is_zero():
    assert oracle.poisson(0.0, 1, 2, 3) == 0
    assert oracle.poisson(-5.0, 1, 2, 3) == 0


def _frame(H=7, W=9, seed=5):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 500, (H, W))


def test_cross_talk_dark_and_adu_closed_form():
    S = _frame()
    H, W = S.shape
    E, A, N = oracle.add_noise(S, 0, seed=1, pattern_seed=2, dark=3.5, xtalk=1e-3, gain=1.7, bias=100.0,
                               saturation=400, poisson=False)
    lam = S + 3.5
    mirror = lam[:, ::-1]
    want = lam + 1e-3 * mirror
    mid = W // 2  # odd width: the middle column has no mirror
    want[:, mid] = lam[:, mid]
    np.testing.assert_allclose(E, want, rtol=1e-15, atol=0)
    adu = np.clip(np.floor(100.0 + want / 1.7 + 0.5), 0, 400)
    assert np.array_equal(A, adu.astype(np.int32))
    np.testing.assert_allclose(N, lam, rtol=0, atol=0)


def test_pixel_response_is_a_fixed_pattern():
    S = np.full((64, 64), 1000.0)
    E1, _, _ = oracle.add_noise(S, 1, seed=10, pattern_seed=99, prnu=0.01, poisson=False)
    E2, _, _ = oracle.add_noise(S, 1, seed=11, pattern_seed=99, prnu=0.01, poisson=False)
    E3, _, _ = oracle.add_noise(S, 1, seed=10, pattern_seed=98, prnu=0.01, poisson=False)
    assert np.array_equal(E1, E2)           # the frame seed does not move the pattern
    assert not np.array_equal(E1, E3)
    r = (E1 / 1000.0 - 1.0).ravel() / 0.01
    assert stats.kstest(r, "norm").pvalue > 1e-4


def test_photon_noise_on_a_flat_field():
    # a flat field of ~40000 e-/px (the level of the paper's aliasing comparison, Fig. 4)
    S = np.full((80, 101), 40000.0)
    E, _, N = oracle.add_noise(S, 0, seed=3, pattern_seed=4, poisson=True)
    d = (N - S).ravel()
    assert abs(d.mean()) < 5 * np.sqrt(40000.0 / d.size)
    assert abs(d.var() / 40000.0 - 1) < 5 * np.sqrt(2.0 / d.size)
    assert np.array_equal(N, np.round(N))
    np.testing.assert_array_equal(E, N)


def test_read_noise_and_determinism():
    S = np.zeros((50, 60))
    E, A, N = oracle.add_noise(S, 2, seed=7, pattern_seed=8, ron=3.0, gain=2.0, bias=1000.0)
    assert not N.any()
    assert stats.kstest(E.ravel() / 3.0, "norm").pvalue > 1e-4
    E2, A2, _ = oracle.add_noise(S, 2, seed=7, pattern_seed=8, ron=3.0, gain=2.0, bias=1000.0)
    assert np.array_equal(E, E2) and np.array_equal(A, A2)
    E3, _, _ = oracle.add_noise(S, 2, seed=8, pattern_seed=8, ron=3.0, gain=2.0, bias=1000.0)
    assert not np.array_equal(E, E3)
