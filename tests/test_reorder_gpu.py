"""Locality order (mds_reorder) and the Phi-term cut-off of the FP32C pass,
on the GPU against the FP64 oracle, through the C ABI.

The cut-off drops the Phi terms of Eq. (2) and Eq. (9) for warp blocks whose
every pair lies at z = delta/sigma >= 8, where log(1/Phi) < 6.3e-16 and
phi/Phi < 5.1e-15; the locality order puts nearby items in the same tile
blocks so that such blocks exist.  Neither may change a result beyond the
stated tolerances, and every array of the API must stay in the caller's item
order: locations, gradients, momenta, injected and Philox draws, held-out
pairs."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG, MDS_ERR_STATE
from gpu_util import TOL, grad_check, scalar_check
from test_parity_gpu import compare, make_model, oracle_ref
from test_cv_gpu import check_fold, make_fold
from test_hmc_gpu import dh_tol

pytestmark = pytest.mark.gpu


def reordered(wl, prec, strip=2, cutoff=None):
    m = make_model(wl, prec, strip=strip)
    m.reorder()
    if cutoff is not None:
        m.set_tail_cutoff(cutoff)
    return m


@pytest.fixture(scope="module")
def paper_workload():
    wl = W.paper_scale()
    return wl, oracle_ref(wl)


def test_paper_scale_far_blocks_and_parity(paper_workload):
    wl, ref = paper_workload
    with make_model(wl, "fp32c") as m:
        far0, total = m.far_blocks()
        m.reorder()
        far1, total1 = m.far_blocks()
        info = compare(m, wl, "fp32c", ref)
        m.set_tail_cutoff(0)
        far_off, _ = m.far_blocks()
        info_off = compare(m, wl, "fp32c", ref)
    print("N=5392 far blocks: unordered", far0, "reordered", far1, "of", total, info, info_off)
    assert total == total1 and far_off == 0
    # the items come in random order, so no block of 64 x 8 pairs is all far;
    # in locality order most are (the mixture's clusters are >= 8 sigma apart)
    assert far0 < 0.02 * total
    assert far1 > 0.5 * total


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,d", [(700, 2), (333, 6), (1000, 3), (129, 5), (65, 1)])
def test_reordered_parity_small_sizes(prec, n, d):
    wl = W.custom(n, d, sigma=0.25, seed=900 + n + d, mixture=(5, 0.3))
    with reordered(wl, prec) as m:
        info = compare(m, wl, prec)
        if prec == "fp32c":
            print(n, d, "far blocks", m.far_blocks(), info)


def test_reorder_keeps_the_caller_order():
    wl = W.custom(500, 3, sigma=0.3, seed=31, mixture=(4, 0.3))
    p = np.random.default_rng(5).standard_normal((wl.n, wl.d))
    with make_model(wl, "fp32c") as a, reordered(wl, "fp32c") as b:
        order = b.get_order()
        assert sorted(order.tolist()) == list(range(wl.n)) and not np.array_equal(order, np.arange(wl.n))
        assert np.array_equal(b.get_locations(), wl.x_eval.astype(np.float64))
        b.set_momentum(p)
        assert np.array_equal(b.get_momentum(), p.astype(np.float32).astype(np.float64))
        la, ga, da = a.gradient()
        lb, gb, db = b.gradient()
    ref = oracle_ref(wl)
    tol = TOL["fp32c"]
    grad_check(gb, ref[2], ref[3][0], tol["g"], s_sq=ref[3][1], u=tol["u"])
    grad_check(ga, ref[2], ref[3][0], tol["g"], s_sq=ref[3][1], u=tol["u"])
    assert math.isclose(la, lb, rel_tol=2e-6) and math.isclose(da, db, rel_tol=2e-5)


def test_reordered_results_are_deterministic():
    wl = W.custom(640, 2, sigma=0.3, seed=32, mixture=(6, 0.3))
    with reordered(wl, "fp32c") as a, reordered(wl, "fp32c") as b:
        la, ga, da = a.gradient()
        lb, gb, db = b.gradient()
    assert la == lb and da == db and np.array_equal(ga, gb)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_reordered_hmc_with_injected_draws_matches_oracle(prec):
    wl = W.custom(300, 2, sigma=0.3, seed=33, mixture=(4, 0.3))
    n_iter, n_steps, eps = 6, 10, 2e-3
    p_all, u_all = W.momenta(34, n_iter, wl.n, wl.d)
    xr, acc_r, dh_r = oracle.hmc(wl.y_packed, wl.x_eval.astype(np.float64), wl.sigma, eps, n_steps, p_all, u_all)
    with reordered(wl, prec) as m:
        ll0, _ = m.log_likelihood()
        acc, dh, _ = m.hmc(n_iter, n_steps, eps, p_all=p_all, u_all=u_all)
        x = m.get_locations()
    tol = dh_tol(prec, ll0)
    for t in range(n_iter):
        if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
            pytest.skip("tie zone")
        assert abs(dh[t] - dh_r[t]) <= tol, (t, dh[t], dh_r[t])
        assert acc[t] == acc_r[t]
    np.testing.assert_allclose(x, xr, rtol=0, atol=(2e-5 if prec == "fp32c" else 1e-11) * (1 + np.abs(xr).max()))


def test_reordered_philox_hmc_matches_oracle():
    wl = W.custom(300, 2, sigma=0.3, seed=35, mixture=(4, 0.3))
    seed, n_iter, n_steps, eps = 78, 5, 10, 2e-3
    p_all = np.zeros((n_iter, wl.n, wl.d))
    u_all = np.zeros(n_iter)
    for t in range(n_iter):
        p, u = oracle.draw_momentum(seed, 0, t, wl.n * wl.d)
        p_all[t] = p.reshape(wl.n, wl.d)
        u_all[t] = u
    xr, acc_r, dh_r = oracle.hmc(wl.y_packed, wl.x_eval.astype(np.float64), wl.sigma, eps, n_steps, p_all, u_all)
    with reordered(wl, "fp32c") as m:
        ll0, _ = m.log_likelihood()
        acc, dh, _ = m.hmc(n_iter, n_steps, eps, seed=seed)
        x = m.get_locations()
    tol = dh_tol("fp32c", ll0) + 1e-5
    for t in range(n_iter):
        if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
            pytest.skip("tie zone")
        assert acc[t] == acc_r[t]
    np.testing.assert_allclose(x, xr, rtol=0, atol=5e-5 * (1 + np.abs(xr).max()))


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_fold_after_reorder_matches_oracle(prec):
    wl = W.custom(420, 2, sigma=0.3, seed=36, mixture=(4, 0.3))
    fold = make_fold(wl.n, 300, 36)
    with reordered(wl, prec) as m:
        m.set_heldout(fold)
        check_fold(m, wl, prec, fold)
        m.lpd_accumulate()
        lpd, draws = m.lpd()
        x = m.get_locations()  # the state as stored (FP32 on the FP32C path)
    uniq = sorted({(min(a, b), max(a, b)) for a, b in fold})
    ref = oracle.lpd(wl.y_packed, uniq, x[None], np.array([wl.sigma]))
    assert draws == 1
    assert lpd == pytest.approx(ref, rel=1e-12, abs=1e-9)


def test_set_data_after_reorder():
    wl = W.custom(380, 2, sigma=0.3, seed=37, mixture=(4, 0.3))
    # new dissimilarities of the same items (same positions and evaluation
    # point, noise scaled by 4/3)
    wl2 = W.custom(380, 2, sigma=0.3, seed=37, noise=0.4, mixture=(4, 0.3))
    assert np.array_equal(wl2.x_eval, wl.x_eval) and not np.array_equal(wl2.y_packed, wl.y_packed)
    with reordered(wl, "fp32c") as m:
        m.set_data(wl2.y_packed)
        ll_r, _ = oracle.loglik(wl2.y_packed, wl.x_eval.astype(np.float64), wl.sigma)
        g_r, s_abs, s_sq = oracle.gradient(wl2.y_packed, wl.x_eval.astype(np.float64), wl.sigma, with_abs=True,
                                           with_sq=True)
        ll, g, _ = m.gradient()
    tol = TOL["fp32c"]
    scalar_check(ll, ll_r, tol["ll"], what="log-likelihood after set_data")
    grad_check(g, g_r, s_abs, tol["g"], s_sq=s_sq, u=tol["u"])


def test_reorder_and_cutoff_errors():
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(200, 2, seed=39)
    with MDS(wl.n, wl.d, "fp32c") as m:
        with pytest.raises(MDSError) as e:
            m.reorder()
        assert e.value.status == MDS_ERR_STATE
        for z in (1.0, 7.9, -1.0, float("inf"), float("nan")):
            with pytest.raises(MDSError) as e:
                m.set_tail_cutoff(z)
            assert e.value.status == MDS_ERR_INVALID_ARG
        m.set_tail_cutoff(0)
        m.set_tail_cutoff(9.5)
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        m.set_heldout([(0, 1)])
        with pytest.raises(MDSError) as e:
            m.reorder()
        assert e.value.status == MDS_ERR_STATE
        m.set_heldout(None)
        m.reorder()
