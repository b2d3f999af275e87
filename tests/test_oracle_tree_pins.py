"""Pins of the phylogenetic-prior oracle (oracle/tree_prior.py, section 2.2)
against things other than itself:

  - the tree covariance V against the paper's path-length definition,
    V_ij = tau0 + [d(root, i) + d(root, j) - d(i, j)] / 2, with d computed by
    networkx shortest paths on the weighted tree;
  - the log density against scipy's matrix-normal log density (with that V);
  - a two-tip tree against the bivariate normal density written out by hand;
  - the gradient against central finite differences of the log density;
  - V against the covariance of tips simulated forward down the tree;
and a set of planted mistakes, each of which must fail at least one pin."""
import math
import types

import networkx as nx
import numpy as np
import pytest
from scipy.stats import matrix_normal

from oracle import tree_prior as TP
from paper_1905_04582_gb300 import workloads as W


def path_length_covariance(forest):
    """V from shortest-path lengths on the weighted forest graph."""
    g = nx.Graph()
    g.add_nodes_from(range(forest.n_nodes))
    for k in range(forest.n_nodes):
        if forest.parent[k] >= 0:
            g.add_edge(k, int(forest.parent[k]), weight=float(forest.length[k]))
    dist = dict(nx.all_pairs_dijkstra_path_length(g))
    roots = {}
    for comp in nx.connected_components(g):
        r = [u for u in comp if forest.parent[u] < 0]
        assert len(r) == 1
        for u in comp:
            roots[u] = r[0]
    n = forest.n
    V = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if roots[i] != roots[j]:
                continue
            r = roots[i]
            if r == i:  # an unsequenced item (a tip that is its own root)
                V[i, j] = forest.tau_u
                continue
            V[i, j] = forest.tau0 + 0.5 * (dist[r][i] + dist[r][j] - dist[i][j])
    return V


def small_forest(seed=3, sizes=(7, 5), lone=2, d=2):
    return W.random_forest(sizes, n_lone=lone, d=d, seed=seed, tau0=0.7, tau_u=1.6)


def args_of(f):
    return (f.parent, f.length, f.sigma_mat, f.mu, f.tau0, f.tau_u)


# --- pins, written against a module-like object M with tree_covariance / logp / gradient


def pin_covariance(M, f):
    V = M.tree_covariance(f.parent, f.length, f.n, f.tau0, f.tau_u)
    np.testing.assert_allclose(V, path_length_covariance(f), rtol=1e-13, atol=1e-13)


def pin_scipy(M, f, x):
    ref = matrix_normal(mean=np.tile(f.mu, (f.n, 1)), rowcov=path_length_covariance(f), colcov=f.sigma_mat).logpdf(x)
    got = M.logp(x, *args_of(f))
    assert math.isclose(got, ref, rel_tol=1e-12, abs_tol=1e-10), (got, ref)


def pin_two_tips(M):
    # root -> tips 0 and 1 with lengths t0, t1, D = 1: bivariate normal with
    # covariance s2 [[tau0 + t0, tau0], [tau0, tau0 + t1]]
    t0, t1, tau0, s2, mu = 0.3, 0.8, 0.5, 1.7, -0.4
    f = W.Forest(2, np.array([2, 2, -1]), np.array([t0, t1, 0.0]), np.array([[s2]]), np.array([mu]), tau0, 9.9)
    x = np.array([[0.25], [-1.1]])
    a, b, c = s2 * (tau0 + t0), s2 * tau0, s2 * (tau0 + t1)
    det = a * c - b * b
    e0, e1 = x[0, 0] - mu, x[1, 0] - mu
    quad = (c * e0 * e0 - 2 * b * e0 * e1 + a * e1 * e1) / det
    ref = -0.5 * quad - math.log(2 * math.pi) - 0.5 * math.log(det)
    got = M.logp(x, *args_of(f))
    assert math.isclose(got, ref, rel_tol=1e-13), (got, ref)
    g = M.gradient(x, *args_of(f))
    g_ref = -np.array([c * e0 - b * e1, a * e1 - b * e0]) / det
    np.testing.assert_allclose(g[:, 0], g_ref, rtol=1e-12)


def pin_finite_differences(M, f, x, h=1e-5):
    g = M.gradient(x, *args_of(f))
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(x.shape[1]):
            xp = x.copy()
            xm = x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd[i, k] = (M.logp(xp, *args_of(f)) - M.logp(xm, *args_of(f))) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def pin_monte_carlo(M, f, draws=6000):
    V = M.tree_covariance(f.parent, f.length, f.n, f.tau0, f.tau_u)
    xs = np.stack([W.brownian_tips(f, seed=1000 + s) for s in range(draws)])  # draws x N x D
    for k in range(f.mu.shape[0]):
        c = np.cov(xs[:, :, k].T)
        ref = V * f.sigma_mat[k, k]
        se = np.sqrt((ref ** 2 + np.outer(np.diag(ref), np.diag(ref))) / draws)  # normal-theory standard error
        assert np.all(np.abs(c - ref) <= 5 * se + 1e-12), np.max(np.abs(c - ref) / (se + 1e-300))


# --- the pins on the oracle


def test_covariance_is_the_path_length_definition():
    for seed in (1, 2, 3):
        pin_covariance(TP, small_forest(seed))


def test_logp_matches_scipy_matrix_normal():
    for seed, d in ((1, 1), (2, 2), (3, 3)):
        f = small_forest(seed, d=d)
        pin_scipy(TP, f, W.brownian_tips(f, seed=seed + 50))


def test_two_tip_closed_form():
    pin_two_tips(TP)


def test_gradient_matches_finite_differences():
    f = small_forest(4, sizes=(9, 4), lone=1, d=2)
    pin_finite_differences(TP, f, W.brownian_tips(f, seed=7))


def test_covariance_matches_forward_simulation():
    f = small_forest(5, sizes=(4, 3), lone=1, d=2)
    pin_monte_carlo(TP, f)


def test_validation_rejects_bad_forests():
    f = small_forest(6)
    bad = f.parent.copy()
    bad[0] = 1  # a tip as parent
    with pytest.raises(ValueError):
        TP.validate(bad, f.length, f.n)
    ln = f.length.copy()
    ln[0] = 0.0
    with pytest.raises(ValueError):
        TP.validate(f.parent, ln, f.n)
    three = f.parent.copy()
    three[f.n - 1] = three[0]  # an unsequenced item joins a node that already has two children
    with pytest.raises(ValueError):
        TP.validate(three, f.length, f.n)


# --- planted mistakes: each must fail a pin


def _mutant(**over):
    m = types.SimpleNamespace(tree_covariance=TP.tree_covariance, logp=TP.logp, gradient=TP.gradient)
    for k, v in over.items():
        setattr(m, k, v)
    return m


def _cov_no_tau0(parent, length, n, tau0, tau_u):
    return TP.tree_covariance(parent, length, n, 0.0, tau_u)


def _cov_depth_sum(parent, length, n, tau0, tau_u):
    V = TP.tree_covariance(parent, length, n, tau0, tau_u)
    dg = np.diag(V).copy()
    return V + 0.25 * (dg[:, None] + dg[None, :]) * (V != 0) * (1 - np.eye(n))


def _logp_drop_logdet_v(x, parent, length, sigma_mat, mu, tau0, tau_u):
    n, d = x.shape
    V = TP.tree_covariance(parent, length, n, tau0, tau_u)
    return TP.logp(x, parent, length, sigma_mat, mu, tau0, tau_u) + 0.5 * d * np.linalg.slogdet(V)[1]


def _logp_logdet_sigma_d(x, parent, length, sigma_mat, mu, tau0, tau_u):
    n, d = x.shape
    return TP.logp(x, parent, length, sigma_mat, mu, tau0, tau_u) + 0.5 * (n - d) * np.linalg.slogdet(sigma_mat)[1]


def _grad_sigma_not_inverted(x, parent, length, sigma_mat, mu, tau0, tau_u):
    n, d = x.shape
    V = TP.tree_covariance(parent, length, n, tau0, tau_u)
    return -np.linalg.solve(V, x - mu[None, :]) @ sigma_mat


def _grad_sign(x, *a):
    return -TP.gradient(x, *a)


def _logp_mean_ignored(x, parent, length, sigma_mat, mu, tau0, tau_u):
    return TP.logp(x, parent, length, sigma_mat, np.zeros_like(mu), tau0, tau_u)


MUTANTS = {
    "root variance dropped": _mutant(tree_covariance=_cov_no_tau0),
    "shared time from depths, not the MRCA": _mutant(tree_covariance=_cov_depth_sum),
    "log|V| term dropped": _mutant(logp=_logp_drop_logdet_v),
    "log|Sigma| weighted by D, not N": _mutant(logp=_logp_logdet_sigma_d),
    "gradient multiplies by Sigma": _mutant(gradient=_grad_sigma_not_inverted),
    "gradient sign": _mutant(gradient=_grad_sign),
    "root mean ignored": _mutant(logp=_logp_mean_ignored),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name):
    M = MUTANTS[name]
    f = small_forest(8, sizes=(6, 5), lone=2, d=2)
    x = W.brownian_tips(f, seed=9)
    pins = [lambda: pin_covariance(M, f), lambda: pin_scipy(M, f, x), lambda: pin_two_tips(M),
            lambda: pin_finite_differences(M, f, x)]
    failed = 0
    for p in pins:
        try:
            p()
        except AssertionError:
            failed += 1
    assert failed > 0, f"mutant '{name}' passes every pin"
