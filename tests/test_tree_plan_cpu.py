"""The work split of the tree prior (host logic, no GPU): every tree is cut
into blocks (whole subtrees of at most ceil(m / 4C) internal nodes) spread
over a cluster of C CTAs and a top (CTA 0).  mds_tree_plan_check builds the
split mds_set_tree_prior would use and verifies it against the forest: each
internal node and tip in exactly one part, child references and levels
consistent, block roots exchanged with matching proxies, buffers in bounds.
Shapes: coalescent forests up to the paper's four subtype trees, the deepest
(caterpillar) and the shallowest (complete) binary trees, many small trees,
unsequenced items, and 60 seeded forests that mix the three ways of joining
lineages."""
import numpy as np
import pytest

from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG
from paper_1905_04582_gb300.mds import tree_plan_check


def heights(f):
    """Height of every tree's root (children before parents by id order is
    not guaranteed, so iterate to a fixed point)."""
    h = np.zeros(len(f.parent), dtype=np.int64)
    changed = True
    while changed:
        changed = False
        for k, p in enumerate(f.parent):
            if p >= 0 and h[p] < h[k] + 1:
                h[p] = h[k] + 1
                changed = True
    return h


@pytest.mark.parametrize("sizes,lone", [((7, 5), 2), ((3, 2), 0), ((300, 200, 90), 10), ((2,) * 40, 7)])
def test_coalescent_forests(sizes, lone):
    f = W.random_forest(sizes, n_lone=lone, d=2, seed=sum(sizes))
    st = tree_plan_check(f.n, f.parent, f.length, 2)
    assert st["trees"] == len(sizes) and st["parts"] == len(sizes) * st["cluster"]
    h = heights(f)
    roots = [k for k in range(f.n, len(f.parent)) if f.parent[k] < 0]
    # the levels of one tree on the chain: its blocks' and its top's, up and down
    assert st["chain_levels"] <= 4 * max(h[r] for r in roots)


def test_paper_forest_uses_full_clusters():
    f = W.random_forest(W.SUBTYPE_SIZES, n_lone=0, d=2, seed=1, rate=0.05)
    st = tree_plan_check(f.n, f.parent, f.length, 2)
    assert st["cluster"] == 8 and st["parts"] == 32
    # each CTA's part stays small: a few tens of KB of shared memory
    assert st["smem_bytes"] < 48 * 1024
    assert st["max_block_nodes"] <= (max(W.SUBTYPE_SIZES) - 1) // 4 + 1


@pytest.mark.parametrize("n", [2, 3, 65, 1000, 3000])
def test_caterpillar(n):
    f = W.ladder_forest(n, d=2, seed=n)
    st = tree_plan_check(f.n, f.parent, f.length, 3)
    # a caterpillar has one level per internal node
    assert st["chain_levels"] == 2 * (n - 1)


@pytest.mark.parametrize("levels", [1, 2, 6, 12])
def test_complete_tree(levels):
    f = W.balanced_forest(levels, d=2, seed=levels)
    st = tree_plan_check(f.n, f.parent, f.length, 2)
    assert st["chain_levels"] == 2 * levels


def test_only_unsequenced_items():
    f = W.random_forest((), n_lone=12, d=2, seed=3)
    st = tree_plan_check(f.n, f.parent, f.length, 2)
    assert st["trees"] == 0 and st["parts"] == 0


def test_not_a_forest_is_rejected():
    f = W.random_forest((6, 4), n_lone=1, d=2, seed=2)
    par = f.parent.copy()
    par[f.n - 1] = par[0]  # an internal node with three children
    with pytest.raises(MDSError) as e:
        tree_plan_check(f.n, par, f.length, 2)
    assert e.value.status == MDS_ERR_INVALID_ARG
    ln = f.length.copy()
    ln[0] = -1.0
    with pytest.raises(MDSError) as e:
        tree_plan_check(f.n, f.parent, ln, 2)
    assert e.value.status == MDS_ERR_INVALID_ARG


def test_random_shapes_and_sizes():
    rng = np.random.default_rng(2024)
    for _ in range(60):
        f = W.mixed_shape_forest(rng)
        n, parent, length = f.n, f.parent, f.length
        d = int(rng.integers(1, 7))
        st = tree_plan_check(n, parent, length, d)
        assert st["parts"] == st["trees"] * st["cluster"]


def test_argument_checks():
    from paper_1905_04582_gb300 import capi
    f = W.random_forest((5, 4), n_lone=1, d=2, seed=4)
    for d in (0, 9):
        with pytest.raises(MDSError) as e:
            tree_plan_check(f.n, f.parent, f.length, d)
        assert e.value.status == MDS_ERR_INVALID_ARG
    st = capi.lib().mds_tree_plan_check(f.n, len(f.parent), None, None, 2, None)
    assert st == MDS_ERR_INVALID_ARG
    with pytest.raises(MDSError) as e:  # fewer nodes than tips
        tree_plan_check(f.n, f.parent[:f.n - 1], f.length[:f.n - 1], 2)
    assert e.value.status == MDS_ERR_INVALID_ARG
