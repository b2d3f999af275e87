"""Single-item random-walk Metropolis (section 2.3's prior-art sampler) on the
GPU against the FP64 oracle, through the C ABI: the same decisions and
log-target differences with injected draws and with the device's Philox
draws, both precisions, in the caller's and the locality order, held-out
pairs left out of the target, a row split over a cluster of CTAs (N > 1024),
the state in global memory (N D beyond shared memory), and the argument
checks.

The FP32C state is FP32, so a proposal x_i + step z is rounded to FP32
before it is evaluated; its reference is a replay at exactly those FP32
points, with each log-target difference taken from two full FP64 oracle
likelihoods.  Tolerance of a difference: a sum of N - 1 differences of terms
of size ~1, each evaluated in FP32 on that path (y - delta and log Phi to a
few ulps): |error| <= 1e-4 (1 + |ref|) (FP64 path, against the oracle's own
sampler: 1e-9).  Decisions are compared outside that tie zone."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG, MDS_ERR_STATE

pytestmark = pytest.mark.gpu

DL_TOL = {"fp32c": 1e-4, "fp64": 1e-9}


def replay_fp32(wl, items, z, u, step, lam=0.0):
    """The FP32C chain evaluated exactly: proposals rounded to FP32 as the
    device forms them (x_i + float(step z)), log-target differences from full
    FP64 likelihoods of the oracle."""
    xs = wl.x_eval.astype(np.float64)
    cur = oracle.loglik(wl.y_packed, xs, wl.sigma)[0]
    acc, dl = [], []
    for t in range(len(items)):
        i = items[t]
        xp = xs.copy()
        xp[i] = (xs[i].astype(np.float32) + (step * np.asarray(z[t])).astype(np.float32)).astype(np.float64)
        new = oracle.loglik(wl.y_packed, xp, wl.sigma)[0]
        a = new - cur - 0.5 * lam * (np.sum(xp[i] ** 2) - np.sum(xs[i] ** 2))
        keep = math.log(u[t]) < a
        acc.append(int(keep))
        dl.append(a)
        if keep:
            xs, cur = xp, new
    return xs, np.array(acc), np.array(dl)


def reference(prec, wl, items, z, u, step, lam=0.0):
    if prec == "fp32c":
        return replay_fp32(wl, items, z, u, step, lam)
    return oracle.rwmh(wl.y_packed, wl.x_eval.astype(np.float64), wl.sigma, step, items, z, u, lam=lam)


def model(wl, prec, reorder=False, lam=0.0):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    m.set_prior(lam)
    if reorder:
        m.reorder()
    return m


def compare_chain(prec, acc, dl, x, acc_r, dl_r, u, xr):
    for t in range(len(u)):
        tol = DL_TOL[prec] * ((1 + abs(dl_r[t])) if prec == "fp32c" else 1.0)
        if abs(math.log(u[t]) - dl_r[t]) <= 2 * tol:
            return t  # tie zone: later states are not comparable
        assert abs(dl[t] - dl_r[t]) <= tol, (t, dl[t], dl_r[t])
        assert acc[t] == acc_r[t], t
    np.testing.assert_allclose(x, xr, rtol=0, atol=(1e-5 if prec == "fp32c" else 1e-12) * (1 + np.abs(xr).max()))
    return len(u)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("reorder", [False, True])
def test_injected_draws_match_oracle(prec, reorder):
    wl = W.custom(300, 2, sigma=0.3, seed=61, mixture=(4, 0.3))
    rng = np.random.default_rng(62)
    k = 300
    items, z, u = rng.integers(0, wl.n, k), rng.standard_normal((k, 2)), rng.uniform(size=k)
    xr, acc_r, dl_r = reference(prec, wl, items, z, u, 0.05, lam=0.1)
    with model(wl, prec, reorder, lam=0.1) as m:
        acc, dl = m.rwmh(k, 0.05, items=items, z_all=z, u_all=u)
        x = m.get_locations()
        ll, _ = m.log_likelihood()  # the pass still agrees with the moved state
    n_ok = compare_chain(prec, acc, dl, x, acc_r, dl_r, u, xr)
    assert n_ok > 100 and 0 < acc_r.sum() < k
    ll_r, _ = oracle.loglik(wl.y_packed, x, wl.sigma)
    assert math.isclose(ll, ll_r, rel_tol=1e-6 if prec == "fp32c" else 1e-11)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_philox_draws_match_oracle(prec):
    wl = W.custom(260, 3, sigma=0.4, seed=63, mixture=(3, 0.3))
    seed, k = 0x5EED_0001_0002, 150
    items, z, u = [], [], []
    for t in range(k):
        i, zz, uu = oracle.rwmh_draws(seed, 0, t, wl.n, wl.d)
        items.append(i)
        z.append(zz)
        u.append(uu)
    items, z, u = np.array(items), np.array(z), np.array(u)
    xr, acc_r, dl_r = reference(prec, wl, items, z, u, 0.04)
    with model(wl, prec) as m:
        acc, dl = m.rwmh(k, 0.04, seed=seed)
        x = m.get_locations()
    assert compare_chain(prec, acc, dl, x, acc_r, dl_r, u, xr) > 50


@pytest.mark.parametrize("prec,n,k", [("fp64", 5000, 300), ("fp32c", 2100, 40)])
def test_cluster_of_ctas_matches_oracle(prec, n, k):
    # N > 1024: the row is split over a cluster of ceil(N / 1024) CTAs whose
    # partial sums meet in every CTA before the decision
    wl = W.custom(n, 2, sigma=0.3, seed=67, mixture=(5, 0.3))
    rng = np.random.default_rng(68)
    items, z, u = rng.integers(0, wl.n, k), rng.standard_normal((k, 2)), rng.uniform(size=k)
    xr, acc_r, dl_r = reference(prec, wl, items, z, u, 0.02, lam=0.05)
    with model(wl, prec, reorder=True, lam=0.05) as m:
        acc, dl = m.rwmh(k, 0.02, items=items, z_all=z, u_all=u)
        x = m.get_locations()
    assert compare_chain(prec, acc, dl, x, acc_r, dl_r, u, xr) > k // 3
    assert 0 < acc_r.sum() < k


def test_state_in_global_memory_matches_oracle():
    # N D FP64 values beyond shared memory: one CTA, X read and written in
    # global memory
    wl = W.custom(12000, 2, sigma=0.3, seed=69, mixture=(6, 0.3))
    rng = np.random.default_rng(70)
    k = 120
    items, z, u = rng.integers(0, wl.n, k), rng.standard_normal((k, 2)), rng.uniform(size=k)
    xr, acc_r, dl_r = reference("fp64", wl, items, z, u, 0.02)
    with model(wl, "fp64") as m:
        acc, dl = m.rwmh(k, 0.02, items=items, z_all=z, u_all=u)
        x = m.get_locations()
    assert compare_chain("fp64", acc, dl, x, acc_r, dl_r, u, xr) > k // 3
    assert 0 < acc_r.sum() < k


def test_held_out_pairs_are_left_out():
    wl = W.custom(200, 2, sigma=0.5, seed=64)
    rng = np.random.default_rng(65)
    iu, ju = np.triu_indices(wl.n, 1)
    pick = rng.choice(len(iu), 800, replace=False)
    fold = np.stack([iu[pick], ju[pick]], 1)
    keep = oracle.keep_mask(wl.n, fold)
    k = 40
    items, z, u = rng.integers(0, wl.n, k), rng.standard_normal((k, 2)), rng.uniform(size=k)
    with model(wl, "fp64") as m:
        m.set_heldout(fold)
        acc, dl = m.rwmh(k, 0.2, items=items, z_all=z, u_all=u)
    xs = wl.x_eval.astype(np.float64)
    for t in range(k):
        xp = xs.copy()
        xp[items[t]] += 0.2 * z[t]
        ref = oracle.loglik(wl.y_packed, xp, wl.sigma, keep=keep)[0] - oracle.loglik(wl.y_packed, xs, wl.sigma,
                                                                                      keep=keep)[0]
        assert abs(dl[t] - ref) <= 1e-9 * (1 + abs(ref)), (t, dl[t], ref)
        if acc[t]:
            xs = xp


def test_argument_checks():
    wl = W.custom(100, 2, seed=66)
    with model(wl, "fp32c") as m:
        with pytest.raises(MDSError) as e:
            m._check(m._lib.mds_rwmh(m._h, 3, 0.1, 0, np.zeros(3, dtype=np.int64).ctypes.data, None, None, None,
                                     None))
        assert e.value.status == MDS_ERR_INVALID_ARG
        with pytest.raises(MDSError) as e:
            m.rwmh(1, 0.1, items=[wl.n], z_all=np.zeros((1, 2)), u_all=[0.5])
        assert e.value.status == MDS_ERR_INVALID_ARG
        with pytest.raises(MDSError) as e:
            m.rwmh(1, -0.1)
        assert e.value.status == MDS_ERR_INVALID_ARG
        f = W.random_forest((60, 40), d=2, seed=1)
        m.set_tree_prior(f.parent, f.length, f.sigma_mat, f.mu, f.tau0, f.tau_u)
        with pytest.raises(MDSError) as e:
            m.rwmh(1, 0.1)
        assert e.value.status == MDS_ERR_STATE
