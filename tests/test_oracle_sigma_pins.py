"""Pins of the oracle's sigma update (the sigma^2 step of the paper's Gibbs
scheme, section 3, with the prior sigma^-2 ~ Gamma(s0, r0) of section 2.2),
independent of the oracle's code:

- with the likelihood switched off the chain must sample the prior: the
  draws of sigma^-2 pass a Kolmogorov-Smirnov test against scipy's Gamma
  (this pins the prior term and the Jacobian of the log-sigma scale);
- one step's decision equals the one computed from scipy's truncated-normal
  log density (Eq. 1) and scipy's Gamma log density plus the log Jacobian;
- the draws (z, u) are standard normal / uniform (KS) and come from the
  Philox4x32-10 block at counter (0, t, chain, 2).
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.distance import pdist

import oracle


def test_prior_only_chain_samples_the_gamma_prior():
    shape, rate = 3.0, 2.0
    rng = np.random.default_rng(0)
    n_iter = 200_000
    z = rng.standard_normal(n_iter)
    u = rng.random(n_iter)
    x = np.zeros((2, 1))
    # the chain in blocks, keeping the last state of each block (thinning by 25)
    s = 0.7
    lam = []
    for b in range(0, n_iter, 25):
        s, _ = oracle.sigma_mh(None, x, s, 0.8, shape, rate, z[b:b + 25], u[b:b + 25], w=0.0)
        lam.append(1.0 / (s * s))
    lam = np.array(lam[200:])
    ks = stats.kstest(lam, stats.gamma(shape, scale=1.0 / rate).cdf)
    assert ks.pvalue > 1e-3, ks
    assert lam.mean() == pytest.approx(shape / rate, rel=0.03)


@pytest.mark.parametrize("z", [0.7, -1.3, 0.05])
def test_single_step_decision_matches_scipy_densities(z):
    rng = np.random.default_rng(1)
    n, d, s, step, s0, r0 = 15, 2, 0.6, 0.4, 2.0, 0.5
    x = rng.standard_normal((n, d))
    y = np.abs(pdist(x) + 0.5 * rng.standard_normal(n * (n - 1) // 2)).astype(np.float32)
    s1 = math.exp(math.log(s) + step * z)
    dl = pdist(x)

    def logpost(sg):
        ll = stats.truncnorm.logpdf(y.astype(np.float64), -dl / sg, np.inf, loc=dl, scale=sg).sum()
        lam = 1.0 / (sg * sg)
        return ll + stats.gamma.logpdf(lam, s0, scale=1.0 / r0) + math.log(2.0 * lam)

    delta = logpost(s1) - logpost(s)
    for f, want in ((0.999, True), (1.001, False)):
        uu = min(math.exp(delta) * f, 0.999999)
        if want is False and math.exp(delta) >= 1.0:
            continue  # always accepted
        s_out, acc = oracle.sigma_mh(y, x, s, step, s0, r0, [z], [uu])
        assert bool(acc[0]) == want
        assert s_out == (s1 if want else s)


def test_sigma_draws_distribution_and_counter():
    zs, us = zip(*(oracle.sigma_draws(0xC0FFEE, 3, t) for t in range(20000)))
    assert stats.kstest(zs, "norm").pvalue > 1e-3
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    o = oracle.philox4x32_10([0, 7, 3, 2], [0xC0FFEE, 0])
    u1, u2 = (o[0] + 0.5) / 2 ** 32, (o[1] + 0.5) / 2 ** 32
    z7, u7 = oracle.sigma_draws(0xC0FFEE, 3, 7)
    assert z7 == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2), rel=1e-14)
    assert u7 == (o[2] + 0.5) / 2 ** 32
