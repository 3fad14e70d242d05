"""Pins for the oracle's seeded Poisson noise (oracle/noise_oracle.c).

The generator is pinned by the known-answer vectors published with its
definition (tests/golden/philox4x32_10_kat.json); the sampler by the Poisson
distribution itself: mean, variance and a chi-square test against the
probability mass function, in both branches (inversion below a mean of 10,
Hormann's transformed rejection from 10 on), plus determinism, independence of
the sample count and dependence on the seed.
"""
import json
import os

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.json")


def test_philox_known_answers(orc):
    for v in json.load(open(GOLDEN))["vectors"]:
        got = orc.philox4x32_10([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert got == [int(x, 16) for x in v["out"]]


@pytest.mark.parametrize("lam", [0.05, 0.7, 3.2, 9.99, 10.0, 17.3, 250.0, 1.0e4, 4.3e5])
def test_poisson_moments_and_distribution(orc, lam):
    n = 400_000
    c = orc.poisson_noise(np.full(n, lam), seed=12345 + int(lam * 7))
    assert np.all(c == np.floor(c)) and np.all(c >= 0)
    mean, var = c.mean(), c.var()
    assert abs(mean - lam) <= 6.0 * np.sqrt(lam / n)
    # the sample variance of a Poisson sample has variance ~ (lam + 2 lam^2) / n
    assert abs(var - lam) <= 6.0 * np.sqrt((lam + 2.0 * lam * lam) / n)
    if lam <= 300:
        lo = int(max(0, np.floor(lam - 6 * np.sqrt(lam) - 2)))
        hi = int(np.ceil(lam + 6 * np.sqrt(lam) + 2))
        ks = np.arange(lo, hi + 1)
        pmf = scipy_stats.poisson.pmf(ks, lam)
        pmf[0] += scipy_stats.poisson.cdf(lo - 1, lam) if lo > 0 else 0.0
        pmf[-1] += scipy_stats.poisson.sf(hi, lam)
        obs = np.array([np.sum(c == k) for k in ks], dtype=float)
        obs[0] += np.sum(c < lo)
        obs[-1] += np.sum(c > hi)
        exp = pmf * n
        keep = exp >= 5.0                    # pool sparse cells into their neighbours' total
        stat = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]) + \
            (obs[~keep].sum() - exp[~keep].sum()) ** 2 / max(exp[~keep].sum(), 1e-300) * (exp[~keep].sum() > 0)
        dof = int(keep.sum()) - 1 + int(exp[~keep].sum() > 0)
        assert scipy_stats.chi2.sf(stat, dof) > 1e-6, (stat, dof)


def test_noise_is_deterministic_and_seeded(orc):
    rng = np.random.default_rng(0)
    chat = rng.uniform(0.0, 2e4, size=(1000, 4))
    chat[::7] = rng.uniform(0.0, 9.0, size=chat[::7].shape)
    chat[3, 2] = 0.0
    a = orc.poisson_noise(chat, seed=99)
    assert np.array_equal(a, orc.poisson_noise(chat, seed=99))
    assert a[3, 2] == 0.0
    # sample i depends on (seed, i, chat[i]) only
    assert np.array_equal(orc.poisson_noise(chat[:100], seed=99), a[:100])
    b = orc.poisson_noise(chat, seed=(99 << 32) | 99)
    assert np.mean(a != b) > 0.9
