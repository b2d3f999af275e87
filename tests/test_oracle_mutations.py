"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that
the pins catch every one: a dropped term, a wrong sign, a wrong index, a
transposed operand, a wrong constant, the half-step drift of the printed
Hamiltonian dynamics, and a wrong Philox multiplier."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.distance import pdist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mds_oracle.c")

MUTANTS = {
    "drop_log_phi": ("return e * e / (2.0 * sigma * sigma) + log_std_normal_cdf(delta / sigma);",
                     "return e * e / (2.0 * sigma * sigma);"),
    "sign_log_phi": ("return e * e / (2.0 * sigma * sigma) + log_std_normal_cdf(delta / sigma);",
                     "return e * e / (2.0 * sigma * sigma) - log_std_normal_cdf(delta / sigma);"),
    "sigma_sq_not_doubled": ("return e * e / (2.0 * sigma * sigma) + log_std_normal_cdf",
                             "return e * e / (sigma * sigma) + log_std_normal_cdf"),
    "row_order_reversed": ("nsum_add(&s, r_term((double)yp[packed_index(n, i, j)]",
                           "nsum_add(&s, r_term((double)yp[i * n - i * (i + 1) / 2 + (n - 1 - j)]"),
    "drop_m_log_sigma": ("*loglik = -m * log(sigma) - sr;", "*loglik = -sr;"),
    "grad_sign": ("nsum_add(&g[k], -term);", "nsum_add(&g[k], term);"),
    "grad_wrong_operand": ("double term = w * (x[i * d + k] - x[j * d + k]) / delta;",
                           "double term = w * (x[i * d + k] - x[j * d + 0]) / delta;"),
    "grad_drop_mills": ("return (delta - y) / (sigma * sigma) + std_normal_pdf(z) / (sigma * std_normal_cdf(z));",
                        "return (delta - y) / (sigma * sigma);"),
    "grad_wrong_y": ("double w = grad_factor(y_at(yp, n, i, j), delta, sigma);",
                     "double w = grad_factor(y_at(yp, n, i, (j + 1) % n == i ? j : (j + 1) % n), delta, sigma);"),
    "dsigma_drop_m": ("*dsigma = -m / sigma + nsum_get(&tot);", "*dsigma = nsum_get(&tot);"),
    "dsigma_sign_mills": ("std_normal_pdf(z) * delta / (sigma * sigma * std_normal_cdf(z));",
                          "-std_normal_pdf(z) * delta / (sigma * sigma * std_normal_cdf(z));"),
    "half_step_drift": ("for (int64_t k = 0; k < nd; ++k) x[k] += eps * p[k];",
                        "for (int64_t k = 0; k < nd; ++k) x[k] += 0.5 * eps * p[k];"),
    "philox_multiplier": ("uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];",
                          "uint64_t p1 = (uint64_t)0xCD9E8D57u * c[1];"),
    "fold_counts_all_pairs": ("if (!keep) return 0.5 * (double)n * (double)(n - 1);",
                              "return 0.5 * (double)n * (double)(n - 1);"),
    "fold_ignored_in_gradient": ("if (j == i || !pair_kept(keep, n, i, j)) continue;", "if (j == i) continue;"),
    "lpd_drop_log_phi": ("- e * e / (2.0 * sigma * sigma) - log_std_normal_cdf(delta / sigma);",
                         "- e * e / (2.0 * sigma * sigma);"),
    "lpd_no_log_S": ("nsum_add(&tot, m + log(e) - log((double)S));", "nsum_add(&tot, m + log(e));"),
    "sigma_prior_no_jacobian": ("return s0 * log(lambda) - r0 * lambda;", "return (s0 - 1.0) * log(lambda) - r0 * lambda;"),
    "sigma_prior_rate_as_scale": ("return s0 * log(lambda) - r0 * lambda;", "return s0 * log(lambda) - lambda / r0;"),
    "sigma_step_on_sigma": ("double s1 = exp(log(s) + step * z_all[t]);", "double s1 = s + step * z_all[t];"),
    "rwmh_difference_reversed": ("dl = w * (row_r(n, d, yp, x, i, x + i * d, sigma) - row_r(n, d, yp, x, i, xi, sigma));",
                                 "dl = w * (row_r(n, d, yp, x, i, xi, sigma) - row_r(n, d, yp, x, i, x + i * d, sigma));"),
    "rwmh_row_skips_a_neighbour": ("        if (j == i) continue;\n        double dd = 0.0;",
                                   "        if (j == i || j == i + 1) continue;\n        double dd = 0.0;"),
    "rwmh_prior_sign": ("double a = dl - 0.5 * lambda * (sq1 - sq0);", "double a = dl + 0.5 * lambda * (sq1 - sq0);"),
}

_i64, _int, _dbl, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
                    "-shared", str(c), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.mdso_loglik.argtypes = [_i64, _int, _vp, _vp, _dbl, _int, _vp, _vp]
    lib.mdso_gradient_rows.argtypes = [_i64, _int, _vp, _vp, _dbl, _vp, _i64, _int, _vp, _vp, _vp]
    lib.mdso_dsigma.argtypes = [_i64, _int, _vp, _vp, _dbl, _int, _vp]
    lib.mdso_leapfrog.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int, _int, _vp, _vp]
    lib.mdso_philox4x32_10.argtypes = [_vp, _vp, _vp]
    lib.mdso_loglik_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _int, _vp, _vp]
    lib.mdso_gradient_rows_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _vp, _i64, _int, _vp, _vp, _vp]
    lib.mdso_lpd.argtypes = [_i64, _int, _vp, _i64, _vp, _int, _vp, _vp, _vp]
    lib.mdso_sigma_mh.argtypes = [_i64, _int, _vp, _vp, _vp, _vp, _dbl, _int, _dbl, _dbl, _dbl, _vp, _vp, _int, _vp]
    lib.mdso_rwmh.argtypes = [_i64, _int, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int, _vp, _vp, _vp, _vp, _vp]
    return lib


def _p(a):
    return a.ctypes.data_as(_vp)


def _pins_hold(lib):
    """The pins of test_oracle_pins.py, condensed; True iff all hold."""
    rng = np.random.default_rng(99)
    n, d, s = 9, 2, 0.7
    x = rng.standard_normal((n, d))
    y = np.abs(pdist(x) + 0.5 * rng.standard_normal(n * (n - 1) // 2)).astype(np.float32)

    def ll(xx, ss=s):
        out = np.zeros(1)
        lib.mdso_loglik(n, d, _p(y), _p(np.ascontiguousarray(xx)), ss, 1, None, _p(out))
        return out[0]

    dl = pdist(x)
    ref = stats.truncnorm.logpdf(y.astype(np.float64), -dl / s, np.inf, loc=dl, scale=s).sum() \
        + 0.5 * len(dl) * math.log(2 * math.pi)
    if not math.isclose(ll(x), ref, rel_tol=1e-12):
        return False
    g = np.zeros((n, d))
    lib.mdso_gradient_rows(n, d, _p(y), _p(x), s, None, 0, 1, _p(g), None, None)
    h = 1e-6
    for i in range(n):
        for k in range(d):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            if not math.isclose(g[i, k], (ll(xp) - ll(xm)) / (2 * h), rel_tol=1e-5, abs_tol=1e-6):
                return False
    ds = np.zeros(1)
    lib.mdso_dsigma(n, d, _p(y), _p(x), s, 1, _p(ds))
    if not math.isclose(ds[0], (ll(x, s + h) - ll(x, s - h)) / (2 * h), rel_tol=1e-6):
        return False
    # a cross-validation fold: training likelihood over the kept pairs, its
    # gradient, and lpd-hat from two draws against scipy's truncated normal
    fold = [(0, 3), (2, 7), (5, 8)]
    keep = np.ones(len(dl), dtype=np.uint8)
    for i, j in fold:
        keep[i * n - i * (i + 1) // 2 + (j - i - 1)] = 0
    kept = keep.astype(bool)
    lk = np.zeros(1)
    lib.mdso_loglik_kept(n, d, _p(y), _p(keep), _p(x), s, 1, None, _p(lk))
    ref = stats.truncnorm.logpdf(y[kept].astype(np.float64), -dl[kept] / s, np.inf, loc=dl[kept], scale=s).sum() \
        + 0.5 * kept.sum() * math.log(2 * math.pi)
    if not math.isclose(lk[0], ref, rel_tol=1e-12):
        return False
    gk = np.zeros((n, d))
    lib.mdso_gradient_rows_kept(n, d, _p(y), _p(keep), _p(x), s, None, 0, 1, _p(gk), None, None)

    def llk(xx):
        out = np.zeros(1)
        lib.mdso_loglik_kept(n, d, _p(y), _p(keep), _p(np.ascontiguousarray(xx)), s, 1, None, _p(out))
        return out[0]
    for i in range(n):
        xp = x.copy(); xp[i, 0] += h
        xm = x.copy(); xm[i, 0] -= h
        if not math.isclose(gk[i, 0], (llk(xp) - llk(xm)) / (2 * h), rel_tol=1e-5, abs_tol=1e-6):
            return False
    pr = np.array(fold, dtype=np.int64)
    xs = np.ascontiguousarray(np.stack([x, x + 0.2]))
    sg = np.array([s, 1.3 * s])
    out = np.zeros(1)
    lib.mdso_lpd(n, d, _p(y), len(fold), _p(pr), 2, _p(xs), _p(sg), _p(out))
    yy = np.array([y[i * n - i * (i + 1) // 2 + (j - i - 1)] for i, j in fold], dtype=np.float64)
    dens = np.zeros((2, len(fold)))
    for t in range(2):
        dd = np.linalg.norm(xs[t][pr[:, 0]] - xs[t][pr[:, 1]], axis=1)
        dens[t] = stats.truncnorm.pdf(yy, -dd / sg[t], np.inf, loc=dd, scale=sg[t])
    if not math.isclose(out[0], np.log(dens.mean(axis=0)).sum(), rel_tol=1e-12):
        return False
    # the sigma update with the likelihood off samples sigma^-2 ~ Gamma(3, 2)
    rs = np.random.default_rng(5)
    zz, uu = rs.standard_normal(60000), rs.random(60000)
    sg = np.array([0.7])
    lam = []
    for b in range(0, 60000, 20):
        lib.mdso_sigma_mh(2, 1, None, None, _p(np.zeros((2, 1))), _p(sg), 0.0, 20, 0.8, 3.0, 2.0,
                          _p(zz[b:b + 20]), _p(uu[b:b + 20]), 1, None)
        lam.append(1.0 / sg[0] ** 2)
    if stats.kstest(lam[100:], stats.gamma(3.0, scale=0.5).cdf).pvalue < 1e-4:
        return False
    # single-item random walk: each log-target difference against full
    # likelihoods; with the likelihood off the chain samples N(0, 1/lambda)
    items = np.array([0, 4, 8, 2, 2], dtype=np.int64)
    zr = np.ascontiguousarray(rng.standard_normal((5, d)))
    ur = np.full(5, 0.5)
    xr = np.ascontiguousarray(x.copy())
    acc = np.zeros(5, dtype=np.int32)
    dlr = np.zeros(5)
    lib.mdso_rwmh(n, d, _p(y), _p(xr), s, 1.0, 0.4, 0.3, 5, _p(items), _p(zr), _p(ur), _p(acc), _p(dlr))
    xs = x.copy()
    for t in range(5):
        xp = xs.copy()
        xp[items[t]] += 0.3 * zr[t]
        ref = ll(xp) - ll(xs) - 0.2 * (np.sum(xp ** 2) - np.sum(xs ** 2))
        if not math.isclose(dlr[t], ref, rel_tol=1e-10, abs_tol=1e-10):
            return False
        if acc[t]:
            xs = xp
    rr = np.random.default_rng(6)
    tot = 60000
    it = np.ascontiguousarray(rr.integers(0, 2, tot).astype(np.int64))
    zz, uu = rr.standard_normal(tot), rr.random(tot)
    xq = np.zeros(2)
    smp = []
    for b in range(0, tot, 20):
        lib.mdso_rwmh(2, 1, None, _p(xq), 1.0, 0.0, 2.0, 1.2, 20, _p(it[b:b + 20]), _p(zz[b:b + 20]),
                      _p(uu[b:b + 20]), None, None)
        smp.append(xq[0])
    if stats.kstest(smp[100:], stats.norm(scale=math.sqrt(0.5)).cdf).pvalue < 1e-4:
        return False
    # harmonic oscillator closed form
    lam, eps, steps = 1.0, 0.1, 5
    xx = rng.standard_normal((4, 2)); pp = rng.standard_normal((4, 2))
    a = np.array([[1 - eps * eps * lam / 2, eps], [-eps * lam * (1 - eps * eps * lam / 4), 1 - eps * eps * lam / 2]])
    an = np.linalg.matrix_power(a, steps)
    x1, p1 = xx.copy(), pp.copy()
    hh = np.zeros(2)
    lib.mdso_leapfrog(4, 2, None, _p(x1), _p(p1), 1.0, 0.0, lam, eps, steps, 1, _p(hh), _p(hh[1:]))
    if not np.allclose(x1, an[0, 0] * xx + an[0, 1] * pp, rtol=1e-12, atol=1e-13):
        return False
    # Philox blocks against a fresh cuRAND host Philox generator (counter (0,0,k,0))
    ref = _curand_blocks(0x0123456789ABCDEF, 4)
    if ref is not None:
        for k in range(4):
            o = np.zeros(4, dtype=np.uint32)
            lib.mdso_philox4x32_10(_p(np.array([0, 0, k, 0], dtype=np.uint32)),
                                   _p(np.array([0x89ABCDEF, 0x01234567], dtype=np.uint32)), _p(o))
            if not np.array_equal(o, ref[4 * k:4 * k + 4]):
                return False
    return True


def _curand_blocks(seed, nblocks):
    try:
        cr = ctypes.CDLL("/usr/local/cuda/lib64/libcurand.so")
    except OSError:
        return None
    gen = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
        return None
    try:
        cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed))
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        cr.curandGenerate(gen, _p(out), ctypes.c_size_t(out.size))
        return out
    finally:
        cr.curandDestroyGenerator(gen)


def test_unmutated_oracle_passes(tmp_path):
    assert _pins_hold(_build(tmp_path, "orig", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not unique"
    assert not _pins_hold(_build(tmp_path, name, text.replace(old, new)))
