"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own code.

- The model of Eq. (1) is a normal truncated to y > 0, so the sum over pairs of
  scipy's truncated-normal log density equals Eq. (2)'s log-likelihood up to
  the dropped (2 pi)^(-M/2) constant: this pins the squared-error term, the
  log Phi truncation term, its sign, the sigma^(-M) factor and the packed
  index of every y_ij.
- The gradient (Eq. (9)) and d/dsigma are pinned by central finite
  differences of the oracle's own likelihood, and at N <= 8 by 50-digit
  numerical differentiation of a brute-force mpmath likelihood that sums the
  truncated-normal density over ordered pairs.
- Invariances: translation / rotation / reflection / permutation.
- The leapfrog integrator is pinned by the closed-form harmonic-oscillator
  map, reversibility and the O(eps^2) energy error; Philox4x32-10 by cuRAND's
  host Philox generator.
"""
import ctypes
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.distance import pdist

import oracle
from paper_1905_04582_gb300 import workloads as W

mpmath = pytest.importorskip("mpmath")


def rand_case(n, d, seed, sigma=0.7, noise=0.5, scale=1.0):
    rng = np.random.default_rng(seed)
    x = scale * rng.standard_normal((n, d))
    y = np.abs(pdist(x) + noise * rng.standard_normal(n * (n - 1) // 2)).astype(np.float32)
    return y, x, sigma


def truncnorm_loglik(y, x, sigma):
    """sum_{i<j} log density of N(delta_ij, sigma^2) truncated to y > 0
    (Eq. (1)), plus (M/2) log(2 pi)."""
    delta = pdist(x)
    a = (0.0 - delta) / sigma
    lp = stats.truncnorm.logpdf(y.astype(np.float64), a, np.inf, loc=delta, scale=sigma)
    return lp.sum() + 0.5 * len(delta) * math.log(2 * math.pi)


@pytest.mark.parametrize("n,d,seed", [(2, 2, 0), (3, 1, 1), (17, 2, 2), (40, 3, 3), (25, 6, 4)])
def test_loglik_equals_truncated_normal_density(n, d, seed):
    y, x, s = rand_case(n, d, seed)
    ll, sr = oracle.loglik(y, x, s)
    ref = truncnorm_loglik(y, x, s)
    assert ll == pytest.approx(ref, rel=1e-12, abs=1e-11)
    m = n * (n - 1) / 2
    assert ll == pytest.approx(-m * math.log(s) - sr, rel=1e-15)


def test_loglik_asymmetric_y_reads_upper_triangle():
    # only the strict upper triangle, i < j, enters (the packed layout)
    y, x, s = rand_case(9, 2, 5)
    full = W.packed_to_full(y, 9)
    full[np.tril_indices(9, -1)] = 123.0  # junk below the diagonal
    assert np.array_equal(W.full_to_packed(full), y)
    ll, _ = oracle.loglik(W.full_to_packed(full), x, s)
    assert ll == pytest.approx(truncnorm_loglik(y, x, s), rel=1e-12)


def fd_grad(y, x, s, h=1e-5):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(x.shape[1]):
            vals = []
            for hh in (h, h / 2):
                xp = x.copy(); xp[i, k] += hh
                xm = x.copy(); xm[i, k] -= hh
                vals.append((oracle.loglik(y, xp, s)[0] - oracle.loglik(y, xm, s)[0]) / (2 * hh))
            g[i, k] = (4 * vals[1] - vals[0]) / 3  # Richardson
    return g


@pytest.mark.parametrize("n,d,seed", [(6, 2, 10), (11, 3, 11), (8, 1, 12)])
def test_gradient_matches_finite_differences(n, d, seed):
    y, x, s = rand_case(n, d, seed)
    g = oracle.gradient(y, x, s)
    fd = fd_grad(y, x, s)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())


def test_dsigma_matches_finite_differences():
    y, x, s = rand_case(12, 2, 13)
    ds = oracle.dsigma(y, x, s)
    vals = []
    for h in (1e-5, 5e-6):
        vals.append((oracle.loglik(y, x, s + h)[0] - oracle.loglik(y, x, s - h)[0]) / (2 * h))
    fd = (4 * vals[1] - vals[0]) / 3
    assert ds == pytest.approx(fd, rel=1e-8)


def mp_loglik(y, x, sigma):
    """Brute force at the caller's mpmath precision: half the sum over ordered
    pairs i != j of the log density of N(delta_ij, sigma^2) truncated to
    (0, inf), written from the density's definition, plus (M/2) log(2 pi)."""
    if True:
        n, d = len(x), len(x[0])
        yf = W.packed_to_full(np.asarray(y, dtype=np.float32), n, dtype=np.float64)
        s = mpmath.mpf(sigma)
        tot = mpmath.mpf(0)
        for i in range(n):
            for j in range(n):
                if i == j:
                    continue
                dl = mpmath.sqrt(mpmath.fsum((x[i][k] - x[j][k]) ** 2 for k in range(d)))
                yy = mpmath.mpf(float(yf[i, j]))
                dens = mpmath.npdf(yy, dl, s) / (1 - mpmath.ncdf(0, dl, s))
                tot += mpmath.log(dens)
        m = n * (n - 1) // 2
        return tot / 2 + m * mpmath.log(2 * mpmath.pi) / 2


@pytest.mark.parametrize("n,d,seed", [(2, 2, 20), (2, 3, 21), (5, 2, 22), (8, 2, 23), (4, 6, 24)])
def test_bruteforce_50_digits(n, d, seed):
    y, x, s = rand_case(n, d, seed)
    with mpmath.workdps(50):
        xm = [[mpmath.mpf(float(v)) for v in row] for row in x]
        ll_mp = mp_loglik(y, xm, s)
    ll, _ = oracle.loglik(y, x, s)
    assert ll == pytest.approx(float(ll_mp), rel=1e-14, abs=1e-13)
    # gradient: 50-digit numerical derivative of the brute-force likelihood
    g = oracle.gradient(y, x, s)
    with mpmath.workdps(50):
        for i in range(n):
            for k in range(d):
                def f(t, i=i, k=k):
                    xx = [row[:] for row in xm]
                    xx[i][k] = t
                    return mp_loglik(y, xx, s)
                ref = mpmath.diff(f, xm[i][k])
                assert g[i, k] == pytest.approx(float(ref), rel=1e-12, abs=1e-12)
        ds_ref = mpmath.diff(lambda t: mp_loglik(y, xm, t), mpmath.mpf(s))
    assert oracle.dsigma(y, x, s) == pytest.approx(float(ds_ref), rel=1e-12)


def test_n2_closed_form_values():
    # N = 2: a single pair, L = log of the truncated normal density at y + log(2 pi)/2
    x = np.array([[0.3, -1.1], [1.4, 0.9]])
    y = np.array([1.7], dtype=np.float32)
    s = 0.4
    dl = math.hypot(1.1, 2.0)
    ref = stats.truncnorm.logpdf(float(y[0]), -dl / s, np.inf, loc=dl, scale=s) + 0.5 * math.log(2 * math.pi)
    assert oracle.loglik(y, x, s)[0] == pytest.approx(ref, rel=1e-13)
    g = oracle.gradient(y, x, s)
    assert np.allclose(g[0], -g[1], rtol=0, atol=1e-14)


def test_translation_rotation_reflection_invariance():
    y, x, s = rand_case(30, 2, 30)
    ll0, _ = oracle.loglik(y, x, s)
    th = 0.77
    r = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    refl = np.array([[1.0, 0.0], [0.0, -1.0]])
    for xt in (x + np.array([3.0, -2.0]), x @ r.T, x @ refl, (x @ r.T) @ refl + 0.5):
        assert oracle.loglik(y, xt, s)[0] == pytest.approx(ll0, rel=1e-12)
    g, a = oracle.gradient(y, x, s, with_abs=True)
    # translation: gradients sum to zero; rotation: total torque is zero
    scale = a.sum(axis=0)
    assert np.all(np.abs(g.sum(axis=0)) <= 1e-12 * scale)
    torque = np.sum(x[:, 0] * g[:, 1] - x[:, 1] * g[:, 0])
    assert abs(torque) <= 1e-12 * np.sum(np.abs(x) * a)


def test_permutation_invariance():
    n = 23
    y, x, s = rand_case(n, 3, 31)
    perm = np.random.default_rng(0).permutation(n)
    full = W.packed_to_full(y, n)
    yp2 = W.full_to_packed(full[np.ix_(perm, perm)])
    ll0, _ = oracle.loglik(y, x, s)
    ll1, _ = oracle.loglik(yp2, x[perm], s)
    assert ll1 == pytest.approx(ll0, rel=1e-13)
    g0 = oracle.gradient(y, x, s)
    g1 = oracle.gradient(yp2, x[perm], s)
    np.testing.assert_allclose(g1, g0[perm], rtol=1e-12, atol=1e-12)


def test_rows_subset_matches_full_gradient():
    y, x, s = rand_case(40, 2, 32)
    g = oracle.gradient(y, x, s)
    rows = np.array([39, 0, 17, 17, 5])
    np.testing.assert_array_equal(oracle.gradient(y, x, s, rows=rows), g[rows])


def test_threads_do_not_change_results():
    y, x, s = rand_case(300, 2, 33)
    assert oracle.loglik(y, x, s, nthreads=1) == oracle.loglik(y, x, s, nthreads=4)
    np.testing.assert_array_equal(oracle.gradient(y, x, s, nthreads=1),
                                  oracle.gradient(y, x, s, nthreads=3))


def test_large_separation_limit():
    # all z = delta / sigma > 40: log Phi = 0 in FP64, so L is the Gaussian part only
    rng = np.random.default_rng(34)
    x = np.arange(10)[:, None] * np.array([[50.0, 0.0]]) + rng.uniform(0, 1, (10, 2))
    s = 1.0
    y = (pdist(x) + rng.standard_normal(45)).astype(np.float32)
    ll, _ = oracle.loglik(y, x, s)
    ref = -np.sum((y.astype(np.float64) - pdist(x)) ** 2) / (2 * s * s)
    assert ll == pytest.approx(ref, rel=1e-14)


def test_coincident_points_reading():
    # x_0 == x_1: that pair contributes delta = 0 to r_01 and nothing to the
    # gradient; central differences of L agree, because |h| is even in h
    rng = np.random.default_rng(35)
    x = rng.standard_normal((5, 2))
    x[1] = x[0]
    y = np.abs(pdist(x) + 0.3).astype(np.float32)
    s = 0.6
    g = oracle.gradient(y, x, s)
    assert np.all(np.isfinite(g))
    np.testing.assert_allclose(g, fd_grad(y, x, s), rtol=1e-7, atol=1e-8)


# ---------------------------------------------------------------- leapfrog


def test_leapfrog_zero_steps_is_identity():
    y, x, s = rand_case(10, 2, 40)
    p = np.random.default_rng(1).standard_normal(x.shape)
    x1, p1, h0, h1 = oracle.leapfrog(y, x, p, s, 1e-2, 0)
    assert np.array_equal(x1, x) and np.array_equal(p1, p) and h0 == h1


@pytest.mark.parametrize("lam,eps,steps", [(1.0, 0.1, 7), (4.0, 0.05, 13), (0.3, 0.5, 3)])
def test_leapfrog_harmonic_oscillator_closed_form(lam, eps, steps):
    # target log pi = -lam/2 ||x||^2: one leapfrog step is the linear map
    # [[1 - eps^2 lam/2, eps], [-eps lam (1 - eps^2 lam/4), 1 - eps^2 lam/2]]
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 3))
    p = rng.standard_normal((6, 3))
    a = np.array([[1 - eps * eps * lam / 2, eps],
                  [-eps * lam * (1 - eps * eps * lam / 4), 1 - eps * eps * lam / 2]])
    an = np.linalg.matrix_power(a, steps)
    x1, p1, h0, h1 = oracle.leapfrog(None, x, p, 1.0, eps, steps, w=0.0, lam=lam)
    np.testing.assert_allclose(x1, an[0, 0] * x + an[0, 1] * p, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(p1, an[1, 0] * x + an[1, 1] * p, rtol=1e-12, atol=1e-13)
    assert h0 == pytest.approx(0.5 * lam * np.sum(x * x) + 0.5 * np.sum(p * p), rel=1e-14)


def test_leapfrog_reversible_on_mds_target():
    y, x, s = rand_case(15, 2, 41)
    p = np.random.default_rng(3).standard_normal(x.shape)
    x1, p1, _, _ = oracle.leapfrog(y, x, p, s, 1e-3, 12)
    x2, p2, _, _ = oracle.leapfrog(y, x1, -p1, s, 1e-3, 12)
    np.testing.assert_allclose(x2, x, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-p2, p, rtol=0, atol=1e-9)


def test_leapfrog_energy_error_is_second_order():
    y, x, s = rand_case(15, 2, 42)
    p = np.random.default_rng(4).standard_normal(x.shape)
    t = 0.02
    errs = []
    for k in (1, 2, 4):
        eps = 2e-3 / k
        _, _, h0, h1 = oracle.leapfrog(y, x, p, s, eps, int(round(t / eps)))
        errs.append(abs(h1 - h0))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_hmc_accept_rule_and_reject_keeps_state():
    # accept iff log u < H0 - H1 (Eq. (8)); a rejected proposal leaves X unchanged
    y, x, s = rand_case(12, 2, 43)
    p_all, _ = W.momenta(5, 1, 12, 2)
    for eps in (0.01, 0.2):
        _, _, dh = oracle.hmc(y, x, s, eps, 5, p_all, np.array([0.5]))
        thr = math.exp(-dh[0])
        if thr < 1.0:
            x_out, acc, _ = oracle.hmc(y, x, s, eps, 5, p_all, np.array([thr * 1.001]))
            assert not acc[0] and np.array_equal(x_out, x)
        x_out, acc, _ = oracle.hmc(y, x, s, eps, 5, p_all, np.array([min(thr, 1.0) * 0.999]))
        assert acc[0] and not np.array_equal(x_out, x)
        x_ref, _, _, _ = oracle.leapfrog(y, x, p_all[0], s, eps, 5)
        np.testing.assert_array_equal(x_out, x_ref)


# ---------------------------------------------------------------- Philox


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    lib = _curand()
    if lib is None:
        pytest.skip("cuRAND not loadable")
    for seed in (0, 0x0123456789ABCDEF, 2**64 - 1):
        gen = ctypes.c_void_p()
        if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
            pytest.skip("cuRAND host Philox generator unavailable")
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            out = np.zeros(4 * 16, dtype=np.uint32)
            assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
        finally:
            lib.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        # a fresh cuRAND host generator hands block k to counter (0, 0, k, 0)
        for k in range(16):
            np.testing.assert_array_equal(oracle.philox4x32_10([0, 0, k, 0], key), out[4 * k:4 * k + 4])


def test_momentum_draws_are_standard_normal():
    p, u = oracle.draw_momentum(1234, 0, 0, 200000)
    assert abs(p.mean()) < 0.01 and abs(p.std() - 1) < 0.01
    assert stats.kstest(p, "norm").pvalue > 1e-3
    assert 0.0 < u < 1.0
    p2, u2 = oracle.draw_momentum(1234, 0, 1, 10)
    assert not np.array_equal(p[:10], p2)
