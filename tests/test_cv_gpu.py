"""Cross-validation folds (section 2.4) on the GPU against the FP64 oracle:
the training likelihood, gradient and dL/dsigma of a fold (held-out pairs
left out, M = the kept pairs), the leapfrog on the fold's target, the lpd-hat
estimator over several draws, and the fold's edge cases (pairs in diagonal
and ragged tiles, a pair given as (j, i), duplicates, clearing the fold,
invalid pairs)."""
import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG, MDS_ERR_STATE
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu


def model(wl, prec, strip=2):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec, strip=strip)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


def make_fold(n, k, seed):
    """k random pairs plus pairs in a diagonal tile, in the last (ragged)
    column block, one given as (j, i), and one duplicate."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    pick = rng.choice(len(iu), size=k, replace=False)
    fold = [(int(iu[p]), int(ju[p])) for p in pick]
    fold += [(1, 2), (3, 60 if n > 60 else n - 1), (n - 1, 0), (5, n - 2)]
    fold += [fold[0]]
    return fold


def check_fold(m, wl, prec, fold):
    keep = oracle.keep_mask(wl.n, fold)
    x64 = m.get_locations().astype(np.float64) if prec == "fp32c" else wl.x_eval.astype(np.float64)
    ll_r, _ = oracle.loglik(wl.y_packed, x64, wl.sigma, keep=keep, nthreads=8)
    g_r, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, wl.sigma, keep=keep, nthreads=8, with_abs=True,
                                       with_sq=True)
    ds_r = oracle.dsigma(wl.y_packed, x64, wl.sigma, keep=keep, nthreads=8)
    ll, g, ds = m.gradient()
    tol = TOL[prec]
    scalar_check(ll, ll_r, tol["ll"], what="fold log-likelihood")
    grad_check(g, g_r, s_abs, tol["g"], s_sq=s_sq, u=tol["u"])
    kept = int(keep.sum())
    scalar_check(ds, ds_r, tol["g"], scale=abs(ds_r) + 2 * kept / wl.sigma, what="fold dL/dsigma")
    return ll, g, ds


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,d,k", [(200, 2, 400), (257, 3, 50), (700, 2, 5000)])
def test_fold_training_likelihood_matches_oracle(prec, n, d, k):
    wl = W.custom(n, d, sigma=0.5, seed=500 + n)
    fold = make_fold(n, k, n)
    with model(wl, prec) as m:
        m.set_heldout(fold)
        assert m.heldout_count() == len({(min(a, b), max(a, b)) for a, b in fold})
        check_fold(m, wl, prec, fold)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_clearing_the_fold_restores_every_pair_bit_for_bit(prec):
    wl = W.custom(300, 2, sigma=0.4, seed=31)
    with model(wl, prec) as a, model(wl, prec) as b:
        ll0, g0, ds0 = a.gradient()
        b.set_heldout(make_fold(300, 300, 2))
        b.gradient()
        b.set_heldout(None)
        assert b.heldout_count() == 0
        ll1, g1, ds1 = b.gradient()
    assert ll0 == ll1 and ds0 == ds1 and np.array_equal(g0, g1)


def test_fold_of_every_pair_gives_zero_likelihood():
    wl = W.custom(70, 2, sigma=0.5, seed=3)
    iu, ju = np.triu_indices(70, 1)
    with model(wl, "fp64") as m:
        m.set_heldout(np.stack([iu, ju], axis=1))
        ll, g, ds = m.gradient()
    assert ll == 0.0 and ds == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_leapfrog_on_fold_target_matches_oracle(prec):
    wl = W.small()
    fold = make_fold(wl.n, 500, 9)
    keep = oracle.keep_mask(wl.n, fold)
    p_all, _ = W.momenta(41, 1, wl.n, wl.d)
    x64 = wl.x_eval.astype(np.float64)
    xr, pr, h0, h1 = oracle.leapfrog(wl.y_packed, x64, p_all[0], wl.sigma, 1e-3, 10, keep=keep)
    with model(wl, prec) as m:
        m.set_heldout(fold)
        dh = m.leapfrog(10, 1e-3, p0=p_all[0])
        x = m.get_locations()
        ll, _ = m.log_likelihood()
    xtol = 2e-6 if prec == "fp32c" else 1e-12
    np.testing.assert_allclose(x, xr, rtol=0, atol=xtol * (1 + np.abs(xr).max()))
    dtol = (2e-6 if prec == "fp32c" else 2e-12) * abs(ll) + (1e-6 if prec == "fp32c" else 1e-12)
    assert abs(dh - (h1 - h0)) <= dtol


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_lpd_over_draws_matches_oracle(prec):
    wl = W.custom(400, 2, sigma=0.5, seed=12)
    fold = make_fold(400, 3000, 13)
    rng = np.random.default_rng(14)
    draws = [wl.x_eval + 0.05 * rng.standard_normal(wl.x_eval.shape) for _ in range(6)]
    sigmas = [0.5, 0.45, 0.55, 0.5, 0.6, 0.4]
    with model(wl, prec) as m:
        m.set_heldout(fold)
        xs = []
        for x, s in zip(draws, sigmas):
            m.set_locations(x)
            m.set_sigma(s)
            m.lpd_accumulate()
            xs.append(m.get_locations())  # the state as stored (FP32 on the FP32C path)
        v, S = m.lpd()
        m.lpd_reset()
        with pytest.raises(MDSError) as ei:
            m.lpd()
        assert ei.value.status == MDS_ERR_STATE
    assert S == 6
    uniq = sorted({(min(a, b), max(a, b)) for a, b in fold})
    ref = oracle.lpd(wl.y_packed, uniq, np.stack(xs), np.array(sigmas))
    assert v == pytest.approx(ref, rel=1e-12, abs=1e-9)


def test_lpd_along_an_hmc_chain():
    """Draws from the device sampler: the lpd of the fold after each HMC
    iteration equals the oracle's estimate over the same states."""
    wl = W.small()
    fold = make_fold(wl.n, 800, 15)
    uniq = sorted({(min(a, b), max(a, b)) for a, b in fold})
    with model(wl, "fp32c") as m:
        m.set_heldout(fold)
        xs = []
        for _ in range(5):
            m.hmc(1, 10, 5e-3, seed=77)
            m.lpd_accumulate()
            xs.append(m.get_locations())
        v, S = m.lpd()
    ref = oracle.lpd(wl.y_packed, uniq, np.stack(xs), wl.sigma)
    assert S == 5 and v == pytest.approx(ref, rel=1e-12, abs=1e-9)


def test_invalid_folds_are_rejected():
    wl = W.custom(50, 2, sigma=0.5, seed=4)
    with model(wl, "fp32c") as m:
        for bad in ([(3, 3)], [(0, 50)], [(-1, 2)]):
            with pytest.raises(MDSError) as ei:
                m.set_heldout(bad)
            assert ei.value.status == MDS_ERR_INVALID_ARG
        with pytest.raises(MDSError) as ei:
            m.lpd_accumulate()  # no fold
        assert ei.value.status == MDS_ERR_STATE
        m.set_heldout([(0, 1)])
        m.set_data(wl.y_packed)  # new data drops the fold
        assert m.heldout_count() == 0
