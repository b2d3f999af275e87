"""Parity of the CUDA pair pass (through the C ABI) with the FP64 CPU oracle:
log-likelihood (Eq. 2), gradient in X (Eq. 9) and dL/dsigma, element by
element on seeded inputs, for both arithmetic paths, at sizes that span
several 64 x 64 tiles with ragged tails, at the paper-scale size N = 5392,
and on the edge cases of the method."""
import math

import numpy as np
import pytest
from scipy.spatial.distance import pdist

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG, MDS_ERR_STATE
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu


def make_model(wl, prec, strip=None, layout="packed"):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec, strip=strip)
    if layout == "packed":
        m.set_data(wl.y_packed)
    else:
        m.set_data(W.packed_to_full(wl.y_packed, wl.n, diag=0.0), layout="full")
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


def oracle_ref(wl, nthreads=8):
    x64 = wl.x_eval.astype(np.float64)
    ll, sr = oracle.loglik(wl.y_packed, x64, wl.sigma, nthreads=nthreads)
    g, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, wl.sigma, nthreads=nthreads, with_abs=True, with_sq=True)
    ds = oracle.dsigma(wl.y_packed, x64, wl.sigma, nthreads=nthreads)
    return ll, sr, g, (s_abs, s_sq), ds


def lg2_floor(wl, prec):
    """Absolute error floor of sum log Phi on the FP32C path: it is taken as
    log2 of per-lane products of 1/Phi (one product per lane half and tile,
    256 per tile), and lg2.approx carries an absolute error of at most
    2^-22.6 per call (PTX ISA), so at most min(M, 256 tiles) calls that hold
    a pair add up to that much each (times ln 2).  It matters only for tiny
    N, where |sum r| itself is small."""
    if prec != "fp32c":
        return 0.0
    nt = (wl.n + 63) // 64
    calls = min(wl.n * (wl.n - 1) // 2, 256 * nt * (nt + 1) // 2)
    return calls * 2.0 ** -22.6 * math.log(2.0)


def compare(m, wl, prec, ref=None):
    ll_ref, sr_ref, g_ref, s_abs, ds_ref = ref if ref is not None else oracle_ref(wl)
    ll, g, ds = m.gradient()
    tol = TOL[prec]
    scalar_check(ll, ll_ref, tol["ll"], what="log-likelihood")
    ll2, sr = m.log_likelihood()
    assert ll2 == ll
    # sum r mixes positive squared errors and negative log Phi terms; the
    # scale for the cancellation rule is their absolute sum
    sq = np.sum((wl.y_packed.astype(np.float64) - pdist(wl.x_eval.astype(np.float64))) ** 2) / (2 * wl.sigma ** 2)
    scalar_check(sr, sr_ref, tol["ll"], scale=sq + abs(sr_ref - sq), what="sum r", abs_floor=lg2_floor(wl, prec))
    info = grad_check(g, g_ref, s_abs[0], tol["g"], s_sq=s_abs[1], u=tol["u"])
    m_pairs = wl.n * (wl.n - 1) / 2
    scale_s = ds_ref + 2 * m_pairs / wl.sigma  # all terms of the sum are >= 0
    scalar_check(ds, ds_ref, tol["g"], scale=scale_s, what="dL/dsigma")
    return info


SMALL = [(2, 2), (3, 1), (17, 2), (64, 2), (65, 3), (130, 2), (200, 2), (333, 6), (700, 2), (257, 8), (129, 5)]


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,d", SMALL)
def test_parity_small_sizes(prec, n, d):
    wl = W.custom(n, d, sigma=0.5, seed=100 + n + d)
    with make_model(wl, prec, strip=2) as m:
        info = compare(m, wl, prec)
    print(prec, n, d, info)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_parity_small_workload(prec):
    wl = W.small()
    with make_model(wl, prec) as m:
        print(prec, compare(m, wl, prec))


@pytest.mark.parametrize("strip", [1, 3, 8])
def test_strip_lengths_agree(strip):
    wl = W.custom(450, 2, sigma=0.4, seed=7, mixture=(3, 0.3))
    ref = oracle_ref(wl)
    with make_model(wl, "fp32c", strip=strip) as m:
        compare(m, wl, "fp32c", ref)


@pytest.fixture(scope="module")
def paper_workload():
    wl = W.paper_scale()
    return wl, oracle_ref(wl)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_parity_paper_scale(prec, paper_workload):
    wl, ref = paper_workload
    with make_model(wl, prec) as m:
        info = compare(m, wl, prec, ref)
    print("N=5392", prec, info)


def test_full_and_packed_layouts_identical():
    wl = W.custom(300, 3, seed=3)
    with make_model(wl, "fp32c", strip=2) as a, make_model(wl, "fp32c", strip=2, layout="full") as b:
        la, ga, da = a.gradient()
        lb, gb, db = b.gradient()
    assert la == lb and da == db and np.array_equal(ga, gb)


def test_device_inputs_match_host_inputs():
    torch = pytest.importorskip("torch")
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(260, 2, seed=4)
    with make_model(wl, "fp32c", strip=2) as a, MDS(wl.n, wl.d, "fp32c", strip=2) as b:
        b.set_data(torch.from_numpy(wl.y_packed).cuda())
        b.set_locations(torch.from_numpy(wl.x_eval).cuda())
        b.set_sigma(wl.sigma)
        out = torch.empty((wl.n, wl.d), dtype=torch.float64, device="cuda")
        lb, _, db = b.gradient(out=out)
        la, ga, da = a.gradient()
    assert la == lb and da == db and np.array_equal(ga, out.cpu().numpy())


def test_repeatable_bitwise():
    wl = W.custom(500, 2, seed=5)
    with make_model(wl, "fp32c", strip=3) as m:
        r1 = m.gradient()
        r2 = m.gradient()
    assert r1[0] == r2[0] and r1[2] == r2[2] and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_coincident_points_and_zero_dissimilarities(prec):
    wl = W.custom(150, 2, seed=6)
    x = wl.x_eval.copy()
    x[10] = x[3]
    x[77] = x[3]
    x[149] = x[0]
    wl.x_eval = x
    y = wl.y_packed.copy()
    y[::17] = 0.0
    wl.y_packed = y
    with make_model(wl, prec, strip=2) as m:
        compare(m, wl, prec)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_large_and_tiny_separations(prec):
    # z = delta/sigma from ~0 (Phi = 1/2) to > 40 (log Phi = 0 in FP64)
    rng = np.random.default_rng(8)
    n = 180
    x = np.concatenate([rng.normal(0, 1e-3, (60, 2)), rng.normal(0, 1.0, (60, 2)),
                        rng.normal(0, 1.0, (60, 2)) + 60.0]).astype(np.float32)
    wl = W.custom(n, 2, sigma=0.5, seed=9)
    wl.x_eval = x
    with make_model(wl, prec, strip=2) as m:
        compare(m, wl, prec)


def test_set_locations_range_error_keeps_state():
    """Locations beyond the FP32C split range are refused on the device before
    anything is written (the set-up kernel derives the split quantum from
    max |x|): INVALID_ARG naming the range, and the previous locations and
    their likelihood unchanged; a NaN entry is INVALID_ARG as well."""
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(120, 2, seed=12)
    with MDS(wl.n, wl.d, "fp32c") as m:
        m.set_data(wl.y_packed)
        m.set_sigma(wl.sigma)
        m.set_locations(wl.x_eval)
        ll0, _ = m.log_likelihood()
        far = wl.x_eval.copy()
        far[7, 0] = 1e36
        with pytest.raises(MDSError) as e:
            m.set_locations(far)
        assert e.value.status == MDS_ERR_INVALID_ARG and "FP32C range" in str(e.value)
        np.testing.assert_array_equal(m.get_locations(dtype=np.float32), wl.x_eval)
        ll1, _ = m.log_likelihood()
        assert ll1 == ll0
        m.set_locations(wl.x_eval)
        assert m.log_likelihood()[0] == ll0
        nanx = wl.x_eval.copy()
        nanx[2, 1] = np.nan
        with pytest.raises(MDSError) as e:
            m.set_locations(nanx)
        assert e.value.status == MDS_ERR_INVALID_ARG


def test_invalid_inputs_are_rejected():
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(100, 2, seed=10)
    with MDS(wl.n, wl.d, "fp32c") as m:
        with pytest.raises(MDSError) as e:
            m.log_likelihood()
        assert e.value.status == MDS_ERR_STATE
        y = wl.y_packed.copy()
        y[W.full_to_packed(np.arange(100 * 100).reshape(100, 100)) == 5 * 100 + 9] = -1.0
        with pytest.raises(MDSError) as e:
            m.set_data(y)
        assert e.value.status == MDS_ERR_INVALID_ARG and "Y(5, 9)" in str(e.value)
        y[0] = np.nan
        with pytest.raises(MDSError):
            m.set_data(y)
        m.set_data(wl.y_packed)
        bad = wl.x_eval.copy()
        bad[3, 1] = np.inf
        with pytest.raises(MDSError):
            m.set_locations(bad)
        with pytest.raises(MDSError):
            m.set_sigma(0.0)
        with pytest.raises(MDSError):
            m.set_sigma(float("nan"))
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        ll, _ = m.log_likelihood()
    ref, _ = oracle.loglik(wl.y_packed, wl.x_eval.astype(np.float64), wl.sigma)
    assert math.isclose(ll, ref, rel_tol=1e-6)


SCALE = [(20000, 2), (20000, 6), (50000, 2), (50000, 6)]


@pytest.mark.slow
@pytest.mark.parametrize("n,d,chunks", [(n, d, None) for n, d in SCALE] +
                         [(20000, 2, ("sm", 1)), (20000, 6, ("sm", 1)), (50000, 6, ("sm", 2))])
def test_parity_scale_sweep_sampled(n, d, chunks):
    """Scale sweep: likelihood and dL/dsigma against the (threaded) oracle,
    gradient on 256 sampled rows computed one by one by the oracle, and the
    translation invariance sum_i grad_i = 0 over all rows.  With `chunks`,
    the shape the benchmark's autotuner picks there (the grouped chunked
    pass) in the locality order, as the benchmark runs it."""
    from paper_1905_04582_gb300.mds import MDS
    wl = W.scale_sweep(n, d)
    x64 = wl.x_eval.astype(np.float64)
    rows = np.random.default_rng(n + d).choice(n, 256, replace=False)
    g_ref, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, wl.sigma, rows=rows, nthreads=16, with_abs=True,
                                         with_sq=True)
    ll_ref, _ = oracle.loglik(wl.y_packed, x64, wl.sigma, nthreads=16)
    ds_ref = oracle.dsigma(wl.y_packed, x64, wl.sigma, nthreads=16)
    with MDS(n, d, "fp32c", chunks=chunks) as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        if chunks is not None:
            m.reorder()
        ll, g, ds = m.gradient()
    tol = TOL["fp32c"]
    scalar_check(ll, ll_ref, tol["ll"], what="log-likelihood")
    scalar_check(ds, ds_ref, tol["g"], scale=ds_ref + n * (n - 1) / wl.sigma, what="dL/dsigma")
    print(n, d, grad_check(g[rows], g_ref, s_abs, tol["g"], s_sq=s_sq, u=tol["u"]))
    tot = np.abs(g).sum(axis=0)
    assert np.all(np.abs(g.sum(axis=0)) <= 1e-5 * tot)
