"""Pins of the oracle's cross-validation functions (section 2.4), independent
of the oracle's own code.

- Training likelihood of a fold: scipy's truncated-normal log density summed
  over the kept pairs only (M = their count); its gradient and d/dsigma by
  50-digit numerical differentiation of a brute-force mpmath likelihood that
  skips the held-out pairs, on N <= 8.
- lpd-hat with one draw: scipy's truncated-normal log density of each
  held-out y (the model of Eq. (1)), summed; with S draws: the log of the
  mean of the 50-digit densities.  The density the estimator uses integrates
  to one over y > 0 (quadrature).
- Degenerate cases: an empty fold changes nothing; holding out every pair
  leaves L = 0; a pair listed as (j, i) is the pair (i, j).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.spatial.distance import pdist

import oracle
from paper_1905_04582_gb300 import workloads as W

mpmath = pytest.importorskip("mpmath")


def rand_case(n, d, seed, sigma=0.7, noise=0.5):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    y = np.abs(pdist(x) + noise * rng.standard_normal(n * (n - 1) // 2)).astype(np.float32)
    return y, x, sigma


def rand_fold(n, k, seed):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    pick = rng.choice(len(iu), size=k, replace=False)
    return np.stack([iu[pick], ju[pick]], axis=1)


def scipy_logdens(y, delta, sigma):
    return stats.truncnorm.logpdf(np.asarray(y, dtype=np.float64), -delta / sigma, np.inf, loc=delta,
                                  scale=sigma)


@pytest.mark.parametrize("n,d,k,seed", [(9, 2, 5, 0), (30, 3, 60, 1), (17, 2, 1, 2)])
def test_training_loglik_is_truncnorm_over_kept_pairs(n, d, k, seed):
    y, x, s = rand_case(n, d, seed)
    fold = rand_fold(n, k, seed + 100)
    keep = oracle.keep_mask(n, fold)
    dl = pdist(x)
    kept = keep.astype(bool)
    ref = scipy_logdens(y[kept], dl[kept], s).sum() + 0.5 * kept.sum() * math.log(2 * math.pi)
    ll, sr = oracle.loglik(y, x, s, keep=keep)
    assert ll == pytest.approx(ref, rel=1e-12, abs=1e-11)
    assert ll == pytest.approx(-kept.sum() * math.log(s) - sr, rel=1e-15)


def mp_loglik_kept(y, x, sigma, heldout):
    """Brute force over ordered pairs i != j, skipping held-out pairs, of the
    truncated-normal log density, halved, plus (M_kept/2) log(2 pi)."""
    n, d = len(x), len(x[0])
    yf = W.packed_to_full(np.asarray(y, dtype=np.float32), n, dtype=np.float64)
    out = {(int(a), int(b)) for a, b in heldout} | {(int(b), int(a)) for a, b in heldout}
    s = mpmath.mpf(sigma)
    tot = mpmath.mpf(0)
    cnt = 0
    for i in range(n):
        for j in range(n):
            if i == j or (i, j) in out:
                continue
            dl = mpmath.sqrt(mpmath.fsum((x[i][k] - x[j][k]) ** 2 for k in range(d)))
            yy = mpmath.mpf(float(yf[i, j]))
            tot += mpmath.log(mpmath.npdf(yy, dl, s) / (1 - mpmath.ncdf(0, dl, s)))
            cnt += 1
    return tot / 2 + (cnt // 2) * mpmath.log(2 * mpmath.pi) / 2


@pytest.mark.parametrize("n,d,seed", [(6, 2, 10), (8, 2, 11), (5, 3, 12)])
def test_training_gradient_and_dsigma_bruteforce_50_digits(n, d, seed):
    y, x, s = rand_case(n, d, seed)
    fold = rand_fold(n, 4, seed)
    fold[0] = fold[0][::-1]  # a pair given as (j, i)
    keep = oracle.keep_mask(n, fold)
    g = oracle.gradient(y, x, s, keep=keep)
    with mpmath.workdps(50):
        xm = [[mpmath.mpf(float(v)) for v in row] for row in x]
        assert oracle.loglik(y, x, s, keep=keep)[0] == pytest.approx(float(mp_loglik_kept(y, xm, s, fold)),
                                                                     rel=1e-14, abs=1e-13)
        for i in range(n):
            for k in range(d):
                def f(t, i=i, k=k):
                    xx = [row[:] for row in xm]
                    xx[i][k] = t
                    return mp_loglik_kept(y, xx, s, fold)
                assert g[i, k] == pytest.approx(float(mpmath.diff(f, xm[i][k])), rel=1e-12, abs=1e-12)
        ds_ref = mpmath.diff(lambda t: mp_loglik_kept(y, xm, t, fold), mpmath.mpf(s))
    assert oracle.dsigma(y, x, s, keep=keep) == pytest.approx(float(ds_ref), rel=1e-12)


def test_empty_fold_and_full_fold():
    y, x, s = rand_case(12, 2, 3)
    n = 12
    ll0 = oracle.loglik(y, x, s)
    assert oracle.loglik(y, x, s, keep=np.ones(n * (n - 1) // 2, np.uint8)) == ll0
    assert oracle.loglik(y, x, s, keep=np.zeros(n * (n - 1) // 2, np.uint8)) == (0.0, 0.0)
    assert np.all(oracle.gradient(y, x, s, keep=np.zeros(n * (n - 1) // 2, np.uint8)) == 0.0)


@pytest.mark.parametrize("sigma", [0.2, 0.7, 3.0])
def test_lpd_single_draw_is_truncnorm_density(sigma):
    y, x, _ = rand_case(20, 2, 4)
    fold = rand_fold(20, 25, 5)
    dl = np.linalg.norm(x[fold[:, 0]] - x[fold[:, 1]], axis=1)
    yy = W.packed_to_full(y, 20, dtype=np.float64)[fold[:, 0], fold[:, 1]]
    ref = scipy_logdens(yy, dl, sigma).sum()
    assert oracle.lpd(y, fold, x, sigma) == pytest.approx(ref, rel=1e-13)


def test_lpd_many_draws_is_log_mean_density_50_digits():
    y, x, _ = rand_case(10, 2, 6)
    fold = rand_fold(10, 7, 7)
    rng = np.random.default_rng(8)
    S = 5
    xs = x[None] + 0.3 * rng.standard_normal((S, 10, 2))
    sig = np.array([0.5, 0.6, 0.4, 0.9, 0.55])
    yf = W.packed_to_full(y, 10, dtype=np.float64)
    with mpmath.workdps(50):
        tot = mpmath.mpf(0)
        for i, j in fold:
            dens = []
            for t in range(S):
                dl = mpmath.sqrt(mpmath.fsum((mpmath.mpf(float(xs[t, i, k])) - mpmath.mpf(float(xs[t, j, k]))) ** 2
                                             for k in range(2)))
                s = mpmath.mpf(float(sig[t]))
                dens.append(mpmath.npdf(mpmath.mpf(float(yf[i, j])), dl, s) / (1 - mpmath.ncdf(0, dl, s)))
            tot += mpmath.log(mpmath.fsum(dens) / S)
    assert oracle.lpd(y, fold, xs, sig) == pytest.approx(float(tot), rel=1e-13)
    # identical draws average to the single-draw value
    assert oracle.lpd(y, fold, np.repeat(xs[:1], 4, axis=0), sig[0]) == pytest.approx(
        oracle.lpd(y, fold, xs[0], sig[0]), rel=1e-14)


@pytest.mark.parametrize("delta,sigma", [(0.0, 1.0), (0.7, 0.3), (2.5, 1.5)])
def test_predictive_density_integrates_to_one(delta, sigma):
    # one held-out pair of an N = 2 problem: exp(lpd) is the density of y
    x = np.array([[0.0, 0.0], [delta, 0.0]])

    def dens(yv):
        return math.exp(oracle.lpd(np.array([yv], dtype=np.float32), [(0, 1)], x, sigma))

    # y is rounded to FP32 before the density is evaluated, hence the tolerance
    tot, err = integrate.quad(dens, 0.0, delta + 12 * sigma, limit=400, points=[delta])
    assert tot == pytest.approx(1.0, abs=2e-6)
