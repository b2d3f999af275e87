"""Plain FP64 oracle of the phylogenetic Brownian-diffusion prior on the
latent locations (section 2.2, the matrix-normal density of X).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing under
``paper_1905_04582_gb300``).

Model.  A forest over the N items: nodes 0..N-1 are the tips (item i is
node i); nodes N.. are internal, each with exactly two children.
parent[k] = -1 marks a root.  length[k] > 0 is the branch length from node k
to its parent (ignored for roots).  A tip that is a root is an "unsequenced"
item.  Brownian motion with D x D covariance Sigma runs down every tree: a
tree's root value is N(mu, tau0 Sigma), a child is N(parent value,
length * Sigma), and an unsequenced item is N(mu, tau_u Sigma) on its own.
Jointly X (N x D) is matrix normal,

    log p(X) = -1/2 tr[Sigma^-1 (X - 1 mu^T)^T V^-1 (X - 1 mu^T)]
               - (N D / 2) log(2 pi) - (N / 2) log|Sigma| - (D / 2) log|V|,

with V the N x N tree covariance: for tips i, j of one tree,
V_ij = tau0 + (elapsed time from the root to their most recent common
ancestor) and V_ii = tau0 + (root-to-tip time); V_ii = tau_u for an
unsequenced item; 0 across trees.  The gradient is
d log p / dX = -V^-1 (X - 1 mu^T) Sigma^-1.

This is the definition written out densely (O(N^2) memory, O(N^3) time): V
from the tips' root paths, then Cholesky factorisations.  It is meant for
N up to a few thousand.
"""
from __future__ import annotations

import numpy as np


def validate(parent, length, n_tips):
    """Check the forest: every internal node has two children, every chain
    of parents ends at a root, lengths are finite and > 0 off the roots.
    Returns (parent, length) as int64 / float64 arrays."""
    parent = np.asarray(parent, dtype=np.int64)
    length = np.asarray(length, dtype=np.float64)
    n_nodes = parent.shape[0]
    if length.shape != (n_nodes,) or n_nodes < n_tips:
        raise ValueError("parent and length need one entry per node, at least N nodes")
    children = np.zeros(n_nodes, dtype=np.int64)
    for k in range(n_nodes):
        p = parent[k]
        if p >= 0:
            if p < n_tips or p >= n_nodes:
                raise ValueError(f"node {k}: parent {p} is not an internal node")
            children[p] += 1
            if not (np.isfinite(length[k]) and length[k] > 0):
                raise ValueError(f"node {k}: branch length must be finite and > 0")
    if np.any(children[n_tips:] != 2):
        raise ValueError("every internal node needs exactly two children")
    for k in range(n_nodes):  # no cycles: every chain reaches a root
        seen, u = 0, k
        while parent[u] >= 0:
            u = parent[u]
            seen += 1
            if seen > n_nodes:
                raise ValueError("the parent links contain a cycle")
    return parent, length


def root_paths(parent, length, n_tips):
    """For every tip: the list of (node, branch length) edges on its path to
    its root, and the root."""
    paths, roots = [], []
    for i in range(n_tips):
        edges, u = [], i
        while parent[u] >= 0:
            edges.append((u, length[u]))
            u = parent[u]
        paths.append(edges)
        roots.append(u)
    return paths, np.array(roots, dtype=np.int64)


def tree_covariance(parent, length, n_tips, tau0, tau_u):
    """V (N x N): tau0 plus the summed lengths of the edges two tips' root
    paths share (the root-to-MRCA time); tau_u on the diagonal of an
    unsequenced item; zero across trees."""
    parent, length = validate(parent, length, n_tips)
    n_nodes = parent.shape[0]
    paths, roots = root_paths(parent, length, n_tips)
    # A[i, e] = 1 where edge e (node e -> parent) lies on tip i's root path
    A = np.zeros((n_tips, n_nodes))
    for i, edges in enumerate(paths):
        for e, _ in edges:
            A[i, e] = 1.0
    V = (A * length[None, :]) @ A.T
    same_tree = roots[:, None] == roots[None, :]
    V = V + tau0 * same_tree
    lone = np.array([parent[i] < 0 for i in range(n_tips)])
    V[lone, :] = 0.0
    V[:, lone] = 0.0
    V[lone, lone] = tau_u
    return V


def _centred(x, mu):
    x = np.asarray(x, dtype=np.float64)
    return x - np.asarray(mu, dtype=np.float64)[None, :]


def logp(x, parent, length, sigma_mat, mu, tau0, tau_u):
    """log p(X | Sigma, tree) of the matrix-normal density (section 2.2)."""
    n, d = np.asarray(x).shape
    V = tree_covariance(parent, length, n, tau0, tau_u)
    S = np.asarray(sigma_mat, dtype=np.float64)
    E = _centred(x, mu)
    Lv = np.linalg.cholesky(V)
    Ls = np.linalg.cholesky(S)
    # tr[S^-1 E^T V^-1 E] = || Lv^-1 E Ls^-T ||_F^2
    W = np.linalg.solve(Lv, E)
    W = np.linalg.solve(Ls, W.T).T
    quad = float(np.sum(W * W))
    logdet_v = 2.0 * float(np.sum(np.log(np.diag(Lv))))
    logdet_s = 2.0 * float(np.sum(np.log(np.diag(Ls))))
    return -0.5 * quad - 0.5 * n * d * np.log(2.0 * np.pi) - 0.5 * n * logdet_s - 0.5 * d * logdet_v


def gradient(x, parent, length, sigma_mat, mu, tau0, tau_u):
    """d log p / dX = -V^-1 (X - 1 mu^T) Sigma^-1 (N x D)."""
    n, d = np.asarray(x).shape
    V = tree_covariance(parent, length, n, tau0, tau_u)
    S = np.asarray(sigma_mat, dtype=np.float64)
    E = _centred(x, mu)
    G = np.linalg.solve(V, E)
    G = np.linalg.solve(S, G.T).T  # Sigma symmetric: (V^-1 E) Sigma^-1
    return -G


# --- HMC with the tree prior in the target (section 2.3 with section 2.2's prior)


def _target(yp, x, sigma, tree):
    """log pi(X) = L(X, sigma) + log p(X | tree) and its gradient, L and dL/dX
    from the serial FP64 oracle of Eq. (2) and (9)."""
    import oracle as O
    ll, _ = O.loglik(yp, x, sigma)
    g = O.gradient(yp, x, sigma)
    return ll + logp(x, *tree), g + gradient(x, *tree)


def leapfrog(yp, x, p, sigma, eps, n_steps, tree):
    """n_steps leapfrog steps of Hamiltonian dynamics with identity mass
    (Eq. (6)-(7), x' = p): half kick, drift, half kick per step.  tree =
    (parent, length, sigma_mat, mu, tau0, tau_u).  Returns (x, p, H0, H1),
    H = -log pi(X) + p^T p / 2."""
    x = np.array(x, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    lp, g = _target(yp, x, sigma, tree)
    h0 = -lp + 0.5 * float(np.sum(p * p))
    for _ in range(n_steps):
        p = p + 0.5 * eps * g
        x = x + eps * p
        lp, g = _target(yp, x, sigma, tree)
        p = p + 0.5 * eps * g
    h1 = -lp + 0.5 * float(np.sum(p * p))
    return x, p, h0, h1


def hmc(yp, x, sigma, eps, n_steps, p_all, u_all, tree):
    """HMC iterations with the given momenta and uniforms: accept the
    trajectory's end point iff log u < H0 - H1 (Eq. (8)).  Returns
    (x, accepted[n_iter], dH[n_iter])."""
    x = np.array(x, dtype=np.float64)
    acc, dh = [], []
    for p0, u in zip(p_all, u_all):
        xn, _, h0, h1 = leapfrog(yp, x, p0, sigma, eps, n_steps, tree)
        keep = bool(np.log(u) < h0 - h1)
        acc.append(int(keep))
        dh.append(h1 - h0)
        if keep:
            x = xn
    return x, np.array(acc, dtype=np.int32), np.array(dh)
