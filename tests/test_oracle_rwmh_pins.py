"""Pins of the single-item random-walk Metropolis oracle (mdso_rwmh, the
prior-art sampler of section 2.3) against things other than itself:

  - every log-target difference equals L(X') - L(X) from the full double
    loop of Eq. (2) (a different code path: all pairs, not one row) plus
    the prior difference;
  - an independent replay of the chain (Python loop, full likelihoods)
    reaches the same decisions and the same final X;
  - with the likelihood off and prior precision lambda the chain samples
    N(0, 1/lambda) in every coordinate (KS test);
  - the Philox draws: items uniform over 0..N-1, z standard normal, u
    uniform (chi-square and KS tests)."""
import math

import numpy as np
from scipy import stats
from scipy.spatial.distance import pdist

import oracle


def _data(n=30, d=2, seed=1, s=0.6):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    y = np.abs(pdist(x) + s * rng.standard_normal(n * (n - 1) // 2)).astype(np.float32)
    return x + 0.1 * rng.standard_normal(x.shape), y, s


def test_differences_are_full_likelihood_differences():
    x, y, s = _data()
    rng = np.random.default_rng(2)
    items = rng.integers(0, x.shape[0], 25)
    z = rng.standard_normal((25, 2))
    u = rng.uniform(size=25)
    lam = 0.3
    xs = x.copy()
    _, acc, dl = oracle.rwmh(y, x, s, 0.2, items, z, u, lam=lam)
    for t in range(25):
        xp = xs.copy()
        xp[items[t]] += 0.2 * z[t]
        ref = oracle.loglik(y, xp, s)[0] - oracle.loglik(y, xs, s)[0] - 0.5 * lam * (np.sum(xp ** 2) - np.sum(xs ** 2))
        assert math.isclose(dl[t], ref, rel_tol=1e-10, abs_tol=1e-10), (t, dl[t], ref)
        if acc[t]:
            xs = xp


def test_independent_replay():
    x, y, s = _data(n=24, seed=3)
    rng = np.random.default_rng(4)
    k = 60
    items, z, u = rng.integers(0, 24, k), rng.standard_normal((k, 2)), rng.uniform(size=k)
    xo, acc, _ = oracle.rwmh(y, x, s, 0.3, items, z, u)
    xs = x.copy()
    cur = oracle.loglik(y, xs, s)[0]
    for t in range(k):
        xp = xs.copy()
        xp[items[t]] += 0.3 * z[t]
        new = oracle.loglik(y, xp, s)[0]
        keep = math.log(u[t]) < new - cur
        assert int(keep) == acc[t]
        if keep:
            xs, cur = xp, new
    np.testing.assert_allclose(xo, xs, rtol=0, atol=1e-14)
    assert 0 < acc.sum() < k


def test_prior_only_chain_samples_the_prior():
    rng = np.random.default_rng(5)
    lam, n, total = 2.0, 3, 90000
    x = np.zeros((n, 1))
    items = rng.integers(0, n, total)
    z, u = rng.standard_normal((total, 1)), rng.uniform(size=total)
    samples = []
    for b in range(0, total, 30):
        x, _, _ = oracle.rwmh(None, x, 1.0, 1.2, items[b:b + 30], z[b:b + 30], u[b:b + 30], w=0.0, lam=lam)
        samples.append(x[0, 0])
    p = stats.kstest(np.array(samples[200:]), stats.norm(scale=1 / math.sqrt(lam)).cdf).pvalue
    assert p > 1e-4, p


def test_philox_draws_have_their_laws():
    n, d, m = 37, 3, 8000
    items, zs, us = [], [], []
    for t in range(m):
        i, z, u = oracle.rwmh_draws(0xDEADBEEF12345, 2, t, n, d)
        items.append(i)
        zs.append(z)
        us.append(u)
    items = np.array(items)
    assert items.min() >= 0 and items.max() < n
    counts = np.bincount(items, minlength=n)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert stats.kstest(np.concatenate(zs), "norm").pvalue > 1e-4
    assert stats.kstest(np.array(us), "uniform").pvalue > 1e-4
