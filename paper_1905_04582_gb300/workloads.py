"""Seeded synthetic inputs shaped like the paper's MDS workloads.

This module only *generates data*: latent positions, the dissimilarity matrix
Y and start points.  It holds none of the likelihood, gradient or HMC
arithmetic, and both the CUDA path's tests/benchmarks and the CPU oracle take
their inputs from it.

The paper's data (5,392 influenza sequences and air-traffic effective
distances, section 3) are not available, so every input here is synthetic:
latent positions from a seeded Gaussian mixture (or a standard normal for the
small case), dissimilarities drawn from the model of Eq. (1) -- the true
distance plus N(0, noise^2) noise, folded at zero so that y_ij >= 0 -- and an
evaluation point X_eval = X_true + N(0, 0.1^2).

Y is returned as the packed strict upper triangle, row-major
(0,1),(0,2),...,(N-2,N-1), in FP32.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.distance import cdist


@dataclass
class Workload:
    name: str
    n: int
    d: int
    sigma: float
    seed: int
    x_true: np.ndarray  # N x D float64
    x_eval: np.ndarray  # N x D float32 (the point the likelihood is evaluated at)
    y_packed: np.ndarray  # N(N-1)/2 float32
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.n * (self.n - 1) // 2


def _positions_normal(rng, n, d):
    return rng.standard_normal((n, d))


def _positions_mixture(rng, n, d, n_comp, spread, box=5.0):
    centres = rng.uniform(-box, box, size=(n_comp, d))
    labels = rng.integers(0, n_comp, size=n)
    return centres[labels] + spread * rng.standard_normal((n, d))


def _packed_dissimilarities(rng, x, noise, block=256):
    """|dist(x_i, x_j) + noise * eps_ij| for i < j, packed row-major, FP32.
    Rows are produced in blocks; the noise stream is drawn in packed order."""
    n = x.shape[0]
    out = np.empty(n * (n - 1) // 2, dtype=np.float32)
    pos = 0
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        dist = cdist(x[i0:i1], x[i0:])  # rows i0..i1-1 against columns i0..N-1
        for r in range(i1 - i0):
            i = i0 + r
            row = dist[r, r + 1:]
            cnt = row.shape[0]
            if cnt == 0:
                continue
            eps = rng.standard_normal(cnt)
            out[pos:pos + cnt] = np.abs(row + noise * eps).astype(np.float32)
            pos += cnt
    assert pos == out.shape[0]
    return out


def make(name, n, d, sigma, seed, noise, mixture=None, eval_jitter=0.1):
    """Build one workload.  mixture=(n_comp, spread) draws positions from a
    Gaussian mixture with centres uniform in [-5, 5]^D; None draws N(0, I)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if mixture is None:
        x_true = _positions_normal(rng, n, d)
    else:
        x_true = _positions_mixture(rng, n, d, mixture[0], mixture[1])
    y = _packed_dissimilarities(rng, x_true, noise)
    x_eval = (x_true + eval_jitter * rng.standard_normal((n, d))).astype(np.float32)
    meta = {"noise_sd": noise, "mixture": mixture, "eval_jitter": eval_jitter}
    return Workload(name, n, d, float(sigma), seed, x_true, x_eval, y, meta)


# --- the five workload recipes ------------------------------------------

def small(seed=0):
    """Oracle-sized case: N=200, D=2, x ~ N(0, I), noise sd 0.5, sigma 0.5."""
    return make("small N=200 D=2", 200, 2, 0.5, seed, 0.5)


def paper_scale(seed=1, d=2):
    """Paper-scale case: N=5392 (the paper's number of items), D=2, 6-component
    mixture (spread 0.3), noise sd 0.3 folded at 0, sigma 0.3."""
    return make(f"paper-scale N=5392 D={d}", 5392, d, 0.3, seed, 0.3, mixture=(6, 0.3))


BATCH_NS = (1600, 1500, 1300, 992)
BATCH_SIGMAS = (0.2, 0.3, 0.4, 0.5)


def batch_datasets():
    """Four independent datasets of uneven N (1600, 1500, 1300, 992), D=2,
    seeds 3..6, 6-component mixtures, noise sd = sigma in {0.2,0.3,0.4,0.5}."""
    return [make(f"batch N={n} D=2", n, 2, s, 3 + k, s, mixture=(6, 0.3))
            for k, (n, s) in enumerate(zip(BATCH_NS, BATCH_SIGMAS))]


def scale_sweep(n, d, seed=7):
    """Scale sweep: N in {20000, 50000}, D in {2, 6}, 12-component mixture,
    noise sd 0.3, sigma 0.3 (Y stored as the packed upper triangle)."""
    return make(f"scale N={n} D={d}", n, d, 0.3, seed, 0.3, mixture=(12, 0.3))


def custom(n, d, sigma=0.5, seed=11, noise=None, mixture=None):
    """Any other size, for tile-edge and ragged-tail tests."""
    return make(f"custom N={n} D={d}", n, d, sigma, seed, sigma if noise is None else noise,
                mixture=mixture)


# --- phylogenetic forests (section 2.2's Brownian-diffusion prior) --------

# the paper's four influenza subtypes (section 3): 1370 + 1389 + 1393 + 1240 = 5392
SUBTYPE_SIZES = (1370, 1389, 1393, 1240)


@dataclass
class Forest:
    n: int                 # tips (items 0..n-1 are nodes 0..n-1)
    parent: np.ndarray     # [n_nodes] int64, -1 for roots
    length: np.ndarray     # [n_nodes] float64 branch length to the parent (0 for roots)
    sigma_mat: np.ndarray  # D x D diffusion covariance
    mu: np.ndarray         # D root mean
    tau0: float            # root variance scalar
    tau_u: float           # variance scalar of unsequenced items (tips that are roots)

    @property
    def n_nodes(self):
        return int(self.parent.shape[0])


def random_forest(tree_sizes, n_lone=0, d=2, seed=0, tau0=1.0, tau_u=2.0, rate=1.0):
    """Random coalescent trees over disjoint groups of items, plus n_lone
    unsequenced items.  Items are assigned to the groups in a seeded random
    order; each tree joins two random lineages at a time after an
    exponential waiting time (rate * k (k - 1) / 2 for k lineages), so branch
    lengths are > 0.  Sigma is a seeded random SPD matrix, mu seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(sum(tree_sizes)) + int(n_lone)
    items = rng.permutation(n)
    parent = [-1] * n
    length = [0.0] * n
    time = [0.0] * n
    pos = 0
    for size in tree_sizes:
        lineages = [int(v) for v in items[pos:pos + size]]
        pos += size
        t = 0.0
        while len(lineages) > 1:
            k = len(lineages)
            t += rng.exponential(1.0 / (rate * k * (k - 1) / 2.0))
            a, b = rng.choice(k, size=2, replace=False)
            u, v = lineages[a], lineages[b]
            node = len(parent)
            parent.append(-1)
            length.append(0.0)
            time.append(t)
            for c in (u, v):
                parent[c] = node
                length[c] = t - time[c]
            lineages = [w for j, w in enumerate(lineages) if j != a and j != b] + [node]
    a = rng.standard_normal((d, d))
    sigma_mat = a @ a.T / d + 0.5 * np.eye(d)
    mu = rng.standard_normal(d)
    return Forest(n, np.array(parent, dtype=np.int64), np.array(length, dtype=np.float64), sigma_mat, mu,
                  float(tau0), float(tau_u))


def _sigma_mu(rng, d):
    a = rng.standard_normal((d, d))
    return a @ a.T / d + 0.5 * np.eye(d), rng.standard_normal(d)


def ladder_forest(n_tips, d=2, seed=0, tau0=1.0, tau_u=2.0):
    """One caterpillar tree (the deepest shape: height n_tips - 1): internal
    node n_tips + k joins the previous internal node (tips 0 and 1 for k = 0)
    and tip k + 1; seeded branch lengths in (0.05, 1.05)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(n_tips)
    parent = np.full(2 * n - 1, -1, dtype=np.int64)
    parent[0] = parent[1] = n
    for k in range(1, n - 1):
        parent[n + k - 1] = n + k
        parent[k + 1] = n + k
    length = 0.05 + rng.uniform(size=2 * n - 1)
    length[-1] = 0.0
    sigma_mat, mu = _sigma_mu(rng, d)
    return Forest(n, parent, length, sigma_mat, mu, float(tau0), float(tau_u))


def balanced_forest(levels, d=2, seed=0, tau0=1.0, tau_u=2.0):
    """One complete binary tree over 2^levels tips (height `levels`): node
    ids by level, tips first; seeded branch lengths in (0.05, 1.05)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 1 << int(levels)
    parent = np.full(2 * n - 1, -1, dtype=np.int64)
    first, width, nxt = 0, n, n
    while width > 1:
        for i in range(width):
            parent[first + i] = nxt + i // 2
        first, nxt, width = nxt, nxt + width // 2, width // 2
    length = 0.05 + rng.uniform(size=2 * n - 1)
    length[-1] = 0.0
    sigma_mat, mu = _sigma_mu(rng, d)
    return Forest(n, parent, length, sigma_mat, mu, float(tau0), float(tau_u))


def mixed_shape_forest(rng, d=2, tau0=1.0, tau_u=2.0):
    """A forest of 1 to 7 trees (1 to 299 tips each) plus up to 4 unsequenced
    items, whose trees join lineages in a random mix of three ways: a random
    pair (coalescent-like), the newest node with a random lineage
    (caterpillar-like), or the two newest (balanced-like).  rng: a numpy
    Generator; branch lengths uniform in (0.05, 1.05); Sigma and mu from rng."""
    sizes = [int(v) for v in rng.integers(1, 300, size=int(rng.integers(1, 8)))]
    n_lone = int(rng.integers(0, 5))
    n = sum(sizes) + n_lone
    items = rng.permutation(n)
    parent = [-1] * n
    pos = 0
    for size in sizes:
        lin = [int(v) for v in items[pos:pos + size]]
        pos += size
        while len(lin) > 1:
            mode = rng.integers(0, 3)
            if mode == 0:
                a, b = rng.choice(len(lin), size=2, replace=False)
            elif mode == 1:
                a, b = len(lin) - 1, int(rng.integers(0, len(lin) - 1))
            else:
                a, b = len(lin) - 1, len(lin) - 2
            u, v = lin[a], lin[b]
            node = len(parent)
            parent.append(-1)
            parent[u] = parent[v] = node
            lin = [w for j, w in enumerate(lin) if j not in (a, b)] + [node]
    parent = np.array(parent, dtype=np.int64)
    length = 0.05 + rng.uniform(size=len(parent))
    length[parent < 0] = 0.0
    sigma_mat, mu = _sigma_mu(rng, d)
    return Forest(n, parent, length, sigma_mat, mu, float(tau0), float(tau_u))


def brownian_tips(forest, seed=0):
    """One draw of X (N x D) from the Brownian diffusion down the forest:
    roots ~ N(mu, tau0 Sigma), children ~ N(parent, length Sigma),
    unsequenced items ~ N(mu, tau_u Sigma)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = forest.mu.shape[0]
    chol = np.linalg.cholesky(forest.sigma_mat)
    n_nodes = forest.n_nodes
    val = np.full((n_nodes, d), np.nan)
    children = [[] for _ in range(n_nodes)]
    for k in range(n_nodes):
        if forest.parent[k] >= 0:
            children[forest.parent[k]].append(k)
    for r in range(n_nodes):
        if forest.parent[r] >= 0:
            continue
        scale = forest.tau_u if r < forest.n else forest.tau0
        val[r] = forest.mu + np.sqrt(scale) * chol @ rng.standard_normal(d)
        stack = [r]
        while stack:
            u = stack.pop()
            for c in children[u]:
                val[c] = val[u] + np.sqrt(forest.length[c]) * chol @ rng.standard_normal(d)
                stack.append(c)
    return val[:forest.n].copy()


# --- layout helpers (pure data movement) ---------------------------------

def packed_to_full(y_packed, n, diag=0.0, dtype=np.float32):
    """Symmetric N x N matrix from the packed strict upper triangle."""
    full = np.zeros((n, n), dtype=dtype)
    iu = np.triu_indices(n, 1)
    full[iu] = y_packed
    full.T[iu] = y_packed
    np.fill_diagonal(full, diag)
    return full


def full_to_packed(full):
    n = full.shape[0]
    return np.ascontiguousarray(full[np.triu_indices(n, 1)])


def momenta(seed, n_iter, n, d):
    """Standard-normal momenta (n_iter x N x D) and Metropolis uniforms
    (n_iter), for runs where both sides are given the same random draws."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.standard_normal((n_iter, n, d))
    u = rng.uniform(size=n_iter)
    return p, u
