"""The chunked FP32C pair pass (chunk_kernel.cu) against the FP64 oracle,
through the C ABI: log-likelihood (Eq. 2), gradient (Eq. 9) and dL/dsigma at
sizes with ragged tails and several dimensions, with chunks that hold one
tile, several row blocks, or a whole problem (segments that start and end
inside a chunk), in the caller's order and in the locality order (far
blocks, measured-cost cuts), at the paper-scale size, with a
cross-validation fold, along HMC trajectories, and the pass-span stamps;
the same in the grouped form (one CTA per SM whose groups of four warps run
the chunks), which sums in the same order as the one-group form."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import capi
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG
from gpu_util import TOL, grad_check, scalar_check
from test_parity_gpu import compare, oracle_ref
from test_cv_gpu import check_fold, make_fold
from test_hmc_gpu import dh_tol

pytestmark = pytest.mark.gpu


def chunked(wl, chunks, reorder=False):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, "fp32c", chunks=chunks)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    if reorder:
        m.reorder()
    return m


SIZES = [(2, 2), (3, 1), (65, 3), (130, 2), (333, 6), (700, 2), (257, 8), (129, 5), (1000, 4)]


@pytest.mark.parametrize("n,d", SIZES)
@pytest.mark.parametrize("chunks", [("count", 1), ("count", 3), ("count", 7), 1, ("sm", 1)])
def test_chunked_parity_small_sizes(n, d, chunks):
    wl = W.custom(n, d, sigma=0.5, seed=100 + n + d)
    with chunked(wl, chunks) as m:
        kind, param, ctas = m.get_pass_shape()
        assert kind in (capi.MDS_PASS_CHUNKS, capi.MDS_PASS_CHUNK_COUNT, capi.MDS_PASS_SM_CHUNKS)
        info = compare(m, wl, "fp32c")
    print(n, d, chunks, ctas, info)


@pytest.mark.parametrize("n,d", [(700, 2), (1000, 3), (333, 6), (2000, 2)])
@pytest.mark.parametrize("chunks", [("count", 5), 1, ("sm", 1), ("sm", 2)])
def test_chunked_parity_locality_order(n, d, chunks):
    wl = W.custom(n, d, sigma=0.25, seed=900 + n + d, mixture=(5, 0.3))
    with chunked(wl, chunks, reorder=True) as m:
        far, total = m.far_blocks()
        info = compare(m, wl, "fp32c")
    print(n, d, chunks, "far", far, "of", total, info)


@pytest.fixture(scope="module")
def paper_workload():
    wl = W.paper_scale()
    return wl, oracle_ref(wl)


@pytest.mark.parametrize("reorder", [False, True])
@pytest.mark.parametrize("chunks", [1, 2, ("sm", 1)])
def test_chunked_parity_paper_scale(paper_workload, reorder, chunks):
    wl, ref = paper_workload
    with chunked(wl, chunks, reorder=reorder) as m:
        info = compare(m, wl, "fp32c", ref)
        kind, param, ctas = m.get_pass_shape()
        far, total = m.far_blocks()
    print("N=5392 chunks", chunks, "reorder", reorder, "ctas", ctas, "far", far, "of", total, info)
    if reorder:
        assert far > 0.5 * total


def test_chunked_and_strip_passes_agree_and_repeat():
    wl = W.custom(1500, 2, sigma=0.3, seed=77, mixture=(6, 0.3))
    ref = oracle_ref(wl)
    from test_parity_gpu import make_model
    with chunked(wl, ("count", 11)) as a, make_model(wl, "fp32c", strip=3) as b:
        la, ga, da = a.gradient()
        la2, ga2, da2 = a.gradient()
        lb, gb, db = b.gradient()
        compare(a, wl, "fp32c", ref)
    # a fixed chunking sums in a fixed order: repeated evaluations are identical
    assert la == la2 and da == da2 and np.array_equal(ga, ga2)
    scalar_check(la, lb, 2e-6, what="chunked vs strip L")


@pytest.mark.parametrize("n,d,k", [(200, 2, 400), (700, 2, 5000), (257, 3, 50)])
@pytest.mark.parametrize("chunks", [("count", 4), ("sm", 1)])
def test_chunked_fold_matches_oracle(n, d, k, chunks):
    wl = W.custom(n, d, sigma=0.5, seed=500 + n)
    fold = make_fold(n, k, n)
    with chunked(wl, chunks) as m:
        m.set_heldout(fold)
        check_fold(m, wl, "fp32c", fold)


@pytest.mark.parametrize("eps", [1.5e-2, 3.5e-2])
@pytest.mark.parametrize("chunks", [("count", 3), ("sm", 1)])
def test_chunked_hmc_injected_draws_match_oracle(eps, chunks):
    wl = W.small()
    n_iter, n_steps = 10, 10
    p_all, u_all = W.momenta(22, n_iter, wl.n, wl.d)
    x64 = wl.x_eval.astype(np.float64)
    xr, acc_r, dh_r = oracle.hmc(wl.y_packed, x64, wl.sigma, eps, n_steps, p_all, u_all)
    with chunked(wl, chunks) as m:
        ll0, _ = m.log_likelihood()
        acc, dh, stats = m.hmc(n_iter, n_steps, eps, p_all=p_all, u_all=u_all)
        x = m.get_locations()
    tol = dh_tol("fp32c", ll0)
    for t in range(n_iter):
        if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
            pytest.skip(f"iteration {t} falls in the tie zone")
        assert abs(dh[t] - dh_r[t]) <= tol, (t, dh[t], dh_r[t])
        assert acc[t] == acc_r[t], (t, dh[t], dh_r[t], u_all[t])
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-5 * (1 + np.abs(xr).max()))


def test_pass_span_stamps_count_every_pass():
    wl = W.custom(3000, 2, sigma=0.3, seed=8, mixture=(6, 0.3))
    with chunked(wl, 1) as m:
        m.gradient()
        m.set_pass_stamps(True)
        m.time_pass(7)
        n, ms = m.get_pass_span()
        # time_pass runs one warm-up pass and 7 timed ones
        assert n == 8, n
        assert 0.0 < ms / n < 50.0, ms
        m.set_pass_stamps(False)
        m.gradient()
        assert m.get_pass_span()[0] == 0


def test_pass_shape_arguments():
    wl = W.custom(300, 2, seed=2)
    from paper_1905_04582_gb300.mds import MDS
    with MDS(wl.n, wl.d, "fp32c") as m, MDS(wl.n, wl.d, "fp64") as m64:
        for kind, param in ((7, 1), (capi.MDS_PASS_STRIPS, -1), (capi.MDS_PASS_CHUNKS, 9),
                            (capi.MDS_PASS_CHUNK_COUNT, 0), (capi.MDS_PASS_SM_CHUNKS, 9)):
            with pytest.raises(MDSError) as ei:
                m.set_pass_shape(kind, param)
            assert ei.value.status == MDS_ERR_INVALID_ARG
        for kind in (capi.MDS_PASS_CHUNKS, capi.MDS_PASS_SM_CHUNKS):
            with pytest.raises(MDSError) as ei:
                m64.set_pass_shape(kind, 1)
            assert ei.value.status == MDS_ERR_INVALID_ARG
        # 300 items: 5 row blocks, 15 tiles, one chunk each; the grouped form
        # runs them as groups of CTAs that each hold one SM's chunk slots
        m.set_pass_shape(capi.MDS_PASS_SM_CHUNKS, 1)
        kind, param, ctas = m.get_pass_shape()
        assert (kind, param) == (capi.MDS_PASS_SM_CHUNKS, 1)
        assert 1 <= ctas <= 15, ctas
        m.set_pass_shape(capi.MDS_PASS_CHUNK_COUNT, 4)
        assert m.get_pass_shape() == (capi.MDS_PASS_CHUNK_COUNT, 4, 4)
        m.set_pass_shape(capi.MDS_PASS_STRIPS, 2)
        assert m.get_pass_shape()[:2] == (capi.MDS_PASS_STRIPS, 2)


@pytest.mark.parametrize("n,d", [(700, 2), (1000, 3), (333, 6)])
def test_grouped_form_sums_in_the_one_group_order(n, d):
    """With no more tiles than chunk slots every chunk is one tile, so the
    grouped and the one-group forms cut the same chunks; each group writes
    its chunk's partial slots, so the results are bitwise those of the
    one-group form."""
    wl = W.custom(n, d, sigma=0.3, seed=40 + n, mixture=(5, 0.3))
    with chunked(wl, 1, reorder=True) as a, chunked(wl, ("sm", 1), reorder=True) as b:
        la, ga, da = a.gradient()
        lb, gb, db = b.gradient()
        ka, kb = a.get_pass_shape(), b.get_pass_shape()
        assert ka[0] == capi.MDS_PASS_CHUNKS and kb[0] == capi.MDS_PASS_SM_CHUNKS
        assert kb[2] < ka[2], (ka, kb)  # fewer, larger CTAs
    assert la == lb and da == db, (la, lb, da, db)
    assert np.array_equal(ga, gb)


def test_grouped_form_paper_scale_repeats_and_agrees(paper_workload):
    """At N = 5392 the grouped form cuts equal-cost pieces per CTA before the
    chunks (its own summation order): repeated evaluations are bitwise
    identical, and it agrees with the one-group form within the stated
    tolerances (both also against the oracle in the parity tests above)."""
    wl, ref = paper_workload
    with chunked(wl, 1, reorder=True) as a, chunked(wl, ("sm", 1), reorder=True) as b:
        la, ga, da = a.gradient()
        lb, gb, db = b.gradient()
        b.set_locations(wl.x_eval)
        lb2, gb2, db2 = b.gradient()
        compare(b, wl, "fp32c", ref)
    assert lb == lb2 and db == db2 and np.array_equal(gb, gb2)
    scalar_check(lb, la, 2e-6, what="grouped vs one-group L")


@pytest.mark.parametrize("n,d,chunks", [(20000, 2, ("count", 8)), (9000, 2, ("count", 8)), (9000, 3, ("count", 4)),
                                        (6000, 6, ("count", 2)), (9000, 2, ("sm", 1))])
def test_chunked_long_runs_are_cut(n, d, chunks):
    """Few large chunks run more than max_seg_tiles(D) tiles (32 at D <= 2,
    16 beyond) in a row block: the pass cuts their row sums into segments of
    at most 64 terms a lane (its second kernel variant) and still matches
    the oracle at the stated tolerances; the grouped case at N = 9000 (chunks
    of about 22 tiles) keeps the uncut loop."""
    wl = W.custom(n, d, sigma=0.3, seed=700 + n + d, mixture=(6, 0.3))
    with chunked(wl, chunks, reorder=True) as m:
        info = compare(m, wl, "fp32c")
    print(n, d, chunks, info)
