"""Batched datasets x chains (one persistent pair-pass launch per step for
all chains) against the FP64 CPU oracle: per-chain likelihood, dL/dsigma and
gradient, and batched HMC with device Philox draws against the oracle's HMC
given the same draws (global chain g keys the stream)."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu


def jitter(x, seed, s=0.05):
    return (x + s * np.random.default_rng(seed).standard_normal(x.shape)).astype(np.float32)


def build(datasets, chains, strip=None):
    from paper_1905_04582_gb300.mds import Batch
    b = Batch([w.n for w in datasets], datasets[0].d, chains, strip=strip)
    xs = []
    for k, (w, c) in enumerate(zip(datasets, chains)):
        b.set_data(k, w.y_packed)
        b.set_sigma(k, w.sigma)
        xs.append([])
        for j in range(c):
            x = jitter(w.x_eval, 1000 * k + j)
            b.set_locations(k, j, x)
            xs[-1].append(x)
    return b, xs


@pytest.mark.parametrize("strip", [1, 2, 4, -8, -32])
def test_batch_evaluate_matches_oracle(strip):
    datasets = [W.custom(300, 2, sigma=0.5, seed=41), W.custom(190, 2, sigma=0.3, seed=42),
                W.custom(65, 2, sigma=0.7, seed=43)]
    chains = [3, 2, 1]
    b, xs = build(datasets, chains, strip=strip)
    with b:
        ll, ds = b.evaluate()
        g = 0
        tol = TOL["fp32c"]
        for k, w in enumerate(datasets):
            for j in range(chains[k]):
                x64 = xs[k][j].astype(np.float64)
                ll_ref, _ = oracle.loglik(w.y_packed, x64, w.sigma)
                ds_ref = oracle.dsigma(w.y_packed, x64, w.sigma)
                g_ref, s_abs, s_sq = oracle.gradient(w.y_packed, x64, w.sigma, with_abs=True, with_sq=True)
                scalar_check(ll[g], ll_ref, tol["ll"], what=f"L chain {g}")
                scalar_check(ds[g], ds_ref, tol["g"], scale=ds_ref + w.n * (w.n - 1) / w.sigma, what=f"dsigma {g}")
                grad_check(b.get_gradient(k, j), g_ref, s_abs, tol["g"], s_sq=s_sq, u=tol["u"], what=f"grad {g}")
                g += 1


def test_batch_uneven_paper_datasets_sampled():
    # the four uneven datasets (N = 1600, 1500, 1300, 992), 8 chains each;
    # two chains per dataset are checked against the oracle
    datasets = W.batch_datasets()
    chains = [8, 8, 8, 8]
    b, xs = build(datasets, chains)
    with b:
        ll, ds = b.evaluate()
        tol = TOL["fp32c"]
        for k, w in enumerate(datasets):
            for j in (0, 7):
                gidx = 8 * k + j
                x64 = xs[k][j].astype(np.float64)
                ll_ref, _ = oracle.loglik(w.y_packed, x64, w.sigma, nthreads=8)
                scalar_check(ll[gidx], ll_ref, tol["ll"], what=f"L chain {gidx}")
                g_ref, s_abs, s_sq = oracle.gradient(w.y_packed, x64, w.sigma, nthreads=8, with_abs=True, with_sq=True)
                grad_check(b.get_gradient(k, j), g_ref, s_abs, tol["g"], s_sq=s_sq, u=tol["u"])


@pytest.mark.parametrize("strip", [None, 2, -16])
def test_batch_hmc_matches_oracle_with_same_draws(strip):
    """Batched HMC (the strip kernel, or every chain's chunked pass as
    concurrent graph branches) against the oracle's HMC with the same draws."""
    datasets = [W.custom(220, 2, sigma=0.5, seed=51), W.custom(130, 2, sigma=0.4, seed=52)]
    chains = [2, 2]
    eps = [1e-2, 1.2e-2]
    n_iter, n_steps, seed = 4, 8, 99
    b, xs = build(datasets, chains, strip=strip)
    with b:
        ll0, _ = b.evaluate()
        acc, dh = b.hmc(n_iter, n_steps, eps, seed=seed)
        g = 0
        for k, w in enumerate(datasets):
            for j in range(chains[k]):
                p_all = np.zeros((n_iter, w.n, w.d))
                u_all = np.zeros(n_iter)
                for t in range(n_iter):
                    p, u = oracle.draw_momentum(seed, g, t, w.n * w.d)
                    p_all[t] = p.reshape(w.n, w.d)
                    u_all[t] = u
                xr, acc_r, dh_r = oracle.hmc(w.y_packed, xs[k][j].astype(np.float64), w.sigma, eps[k], n_steps,
                                             p_all, u_all)
                tol = 2e-6 * abs(ll0[g]) + 1e-5
                for t in range(n_iter):
                    if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
                        pytest.skip("tie zone")
                    assert acc[t, g] == acc_r[t], (g, t, dh[t, g], dh_r[t])
                    assert abs(dh[t, g] - dh_r[t]) <= tol, (g, t, dh[t, g], dh_r[t])
                x = b.get_locations(k, j)
                np.testing.assert_allclose(x, xr, rtol=0, atol=5e-5 * (1 + np.abs(xr).max()))
                g += 1


@pytest.mark.parametrize("strip", [2, -6])
def test_batch_reorder_matches_oracle(strip):
    """mds_batch_reorder: each dataset's Y repacked once in the locality order
    of its first chain, every chain adopting it (the far blocks then skip the
    Phi terms in the chunked shape); every chain's L, gradient and dL/dsigma
    against the oracle in the caller's item order, and the locations read
    back unchanged."""
    datasets = [W.custom(700, 2, sigma=0.3, seed=61, mixture=(5, 0.3)),
                W.custom(450, 2, sigma=0.25, seed=62, mixture=(4, 0.3))]
    chains = [3, 2]
    b, xs = build(datasets, chains, strip=strip)
    with b:
        b.reorder()
        ll, ds = b.evaluate()
        g = 0
        tol = TOL["fp32c"]
        for k, w in enumerate(datasets):
            for j in range(chains[k]):
                np.testing.assert_array_equal(b.get_locations(k, j), xs[k][j])
                x64 = xs[k][j].astype(np.float64)
                ll_ref, _ = oracle.loglik(w.y_packed, x64, w.sigma)
                ds_ref = oracle.dsigma(w.y_packed, x64, w.sigma)
                g_ref, s_abs, s_sq = oracle.gradient(w.y_packed, x64, w.sigma, with_abs=True, with_sq=True)
                scalar_check(ll[g], ll_ref, tol["ll"], what=f"L chain {g}")
                scalar_check(ds[g], ds_ref, tol["g"], scale=ds_ref + w.n * (w.n - 1) / w.sigma, what=f"dsigma {g}")
                grad_check(b.get_gradient(k, j), g_ref, s_abs, tol["g"], s_sq=s_sq, u=tol["u"], what=f"grad {g}")
                g += 1


def test_batch_reorder_hmc_matches_oracle():
    datasets = [W.custom(400, 2, sigma=0.4, seed=71, mixture=(4, 0.3)), W.custom(260, 2, sigma=0.35, seed=72)]
    chains = [2, 2]
    eps = [5e-3, 6e-3]
    n_iter, n_steps, seed = 3, 8, 17
    b, xs = build(datasets, chains, strip=-6)
    with b:
        b.reorder()
        ll0, _ = b.evaluate()
        acc, dh = b.hmc(n_iter, n_steps, eps, seed=seed)
        g = 0
        for k, w in enumerate(datasets):
            for j in range(chains[k]):
                p_all = np.zeros((n_iter, w.n, w.d))
                u_all = np.zeros(n_iter)
                for t in range(n_iter):
                    p, u = oracle.draw_momentum(seed, g, t, w.n * w.d)
                    p_all[t] = p.reshape(w.n, w.d)
                    u_all[t] = u
                xr, acc_r, dh_r = oracle.hmc(w.y_packed, xs[k][j].astype(np.float64), w.sigma, eps[k], n_steps,
                                             p_all, u_all)
                tol = 2e-6 * abs(ll0[g]) + 1e-5
                for t in range(n_iter):
                    if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
                        pytest.skip("tie zone")
                    assert acc[t, g] == acc_r[t], (g, t, dh[t, g], dh_r[t])
                    assert abs(dh[t, g] - dh_r[t]) <= tol, (g, t, dh[t, g], dh_r[t])
                np.testing.assert_allclose(b.get_locations(k, j), xr, rtol=0, atol=5e-5 * (1 + np.abs(xr).max()))
                g += 1
