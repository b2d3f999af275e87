"""The sigma update (section 3's sigma^2 step; random walk on log sigma with
the Gamma prior on sigma^-2) on the GPU against the FP64 oracle: the same
decisions and final sigma for injected draws and for the device's Philox
draws (outside the tie zone set by the stated likelihood error), the state
after accepted and rejected proposals, and HMC after sigma moved (the
captured graph is updated in place)."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu


def model(wl, prec, strip=2):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec, strip=strip)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


def oracle_chain(wl, x, sigma, step, shape, rate, z, u):
    """The oracle's decisions, plus for each step whether it sits in the tie
    zone |log u - (P' - P)| <= 4 tol |L| (FP32C: tol = 1e-6)."""
    s = sigma
    acc = []
    ties = []
    for t in range(len(z)):
        s1 = math.exp(math.log(s) + step * z[t])
        l0, _ = oracle.loglik(wl.y_packed, x, s, nthreads=8)
        l1, _ = oracle.loglik(wl.y_packed, x, s1, nthreads=8)
        p0 = l0 + shape * math.log(1 / s ** 2) - rate / s ** 2
        p1 = l1 + shape * math.log(1 / s1 ** 2) - rate / s1 ** 2
        ties.append(abs(math.log(u[t]) - (p1 - p0)) <= 4e-6 * (abs(l0) + abs(l1)))
        s_o, a = oracle.sigma_mh(wl.y_packed, x, s, step, shape, rate, [z[t]], [u[t]], nthreads=8)
        acc.append(bool(a[0]))
        s = s_o
    return s, np.array(acc), np.array(ties)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_injected_draws_match_oracle(prec):
    wl = W.small()
    rng = np.random.default_rng(3)
    n = 12
    z, u = rng.standard_normal(n), rng.random(n)
    step, shape, rate = 0.05, 2.0, 0.5
    with model(wl, prec) as m:
        x = m.get_locations()
        acc, s = m.sigma_mh(n, step, shape, rate, z_all=z, u_all=u)
    s_ref, acc_ref, ties = oracle_chain(wl, x, wl.sigma, step, shape, rate, z, u)
    first_tie = int(np.argmax(ties)) if ties.any() else n
    assert np.array_equal(acc[:first_tie], acc_ref[:first_tie])
    if first_tie == n:
        assert s == pytest.approx(s_ref, rel=1e-14)
    assert 0 < acc.sum() < n  # both branches exercised


def test_device_philox_draws_match_oracle():
    wl = W.small()
    seed, n, step, shape, rate = 0xABCDEF12345, 10, 0.05, 2.0, 0.5
    zu = [oracle.sigma_draws(seed, 0, t) for t in range(2 * n)]
    with model(wl, "fp64") as m:
        x = m.get_locations()
        acc1, s1 = m.sigma_mh(n, step, shape, rate, seed=seed)
        acc2, s2 = m.sigma_mh(n, step, shape, rate, seed=seed)  # continues the stream
    z = np.array([a for a, _ in zu])
    u = np.array([b for _, b in zu])
    s_ref, acc_ref, ties = oracle_chain(wl, x, wl.sigma, step, shape, rate, z, u)
    acc = np.concatenate([acc1, acc2])
    first_tie = int(np.argmax(ties)) if ties.any() else 2 * n
    assert np.array_equal(acc[:first_tie], acc_ref[:first_tie])
    if first_tie == 2 * n:
        assert s2 == pytest.approx(s_ref, rel=1e-14)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_state_after_updates_and_hmc_after_sigma_moved(prec):
    """After accepted and rejected proposals the cached pass is consistent with
    the current sigma, and an HMC iteration run after sigma moved (graph
    updated in place) matches the oracle's leapfrog at the new sigma."""
    wl = W.small()
    with model(wl, prec) as m:
        m.hmc(1, 5, 1e-3, seed=1)  # a captured graph exists
        acc, s = m.sigma_mh(2, 0.3, 2.0, 0.5, z_all=[1.0, 50.0], u_all=[0.5, 0.5])
        assert acc[1] == False  # a step of 15 in log sigma is rejected
        x = m.get_locations()
        ll, g, ds = m.gradient()
        x64 = x.astype(np.float64)
        ll_r, _ = oracle.loglik(wl.y_packed, x64, s, nthreads=8)
        g_r, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, s, nthreads=8, with_abs=True, with_sq=True)
        tol = TOL[prec]
        scalar_check(ll, ll_r, tol["ll"], what="L after sigma updates")
        grad_check(g, g_r, s_abs, tol["g"], s_sq=s_sq, u=tol["u"])
        p_all, u_all = W.momenta(5, 1, wl.n, wl.d)
        xr, _, _ = oracle.hmc(wl.y_packed, x64, s, 1e-3, 10, p_all, np.array([0.5]))
        m.hmc(1, 10, 1e-3, p_all=p_all, u_all=np.array([0.5]))
        xg = m.get_locations()
    xtol = 2e-6 if prec == "fp32c" else 1e-12
    np.testing.assert_allclose(xg, xr, rtol=0, atol=xtol * (1 + np.abs(xr).max()))
