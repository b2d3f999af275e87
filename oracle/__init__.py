"""ctypes loader for the serial FP64 CPU oracle (``mds_oracle.c``).

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` leg and
reference arm, never by the library under ``paper_1905_04582_gb300``.

Every function takes numpy arrays and returns numpy arrays / floats.  Y is
always the packed strict upper triangle (row-major (0,1),(0,2),...,(N-2,N-1))
in FP32, X is FP64 (FP32 locations are widened exactly by the caller).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mds_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmds_oracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.mdso_loglik_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _int, _vp, _vp]
            lib.mdso_gradient_rows_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _vp, _i64, _int, _vp,
                                                    _vp, _vp]
            lib.mdso_dsigma_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _int, _vp]
            lib.mdso_leapfrog_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _vp, _dbl, _dbl, _dbl, _dbl,
                                               _int, _int, _vp, _vp]
            lib.mdso_hmc_kept.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int, _int,
                                          _vp, _vp, _int, _vp, _vp]
            lib.mdso_lpd.argtypes = [_i64, _int, _vp, _i64, _vp, _int, _vp, _vp, _vp]
            lib.mdso_sigma_mh.argtypes = [_i64, _int, _vp, _vp, _vp, _vp, _dbl, _int, _dbl, _dbl, _dbl, _vp,
                                          _vp, _int, _vp]
            lib.mdso_sigma_draws.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             _vp, _vp]
            lib.mdso_sigma_draws.restype = None
            lib.mdso_philox4x32_10.argtypes = [_vp, _vp, _vp]
            lib.mdso_rwmh.argtypes = [_i64, _int, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int, _vp, _vp, _vp, _vp, _vp]
            lib.mdso_rwmh.restype = _int
            lib.mdso_rwmh_draws.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                            _i64, _int, _vp, _vp, _vp]
            lib.mdso_rwmh_draws.restype = None
            lib.mdso_draw_momentum.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, _i64, _vp, _vp]
            for f in ("mdso_loglik_kept", "mdso_gradient_rows_kept", "mdso_dsigma_kept",
                      "mdso_leapfrog_kept", "mdso_hmc_kept", "mdso_lpd", "mdso_sigma_mh"):
                getattr(lib, f).restype = _int
            lib.mdso_philox4x32_10.restype = None
            lib.mdso_draw_momentum.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _prep(yp, x):
    yp = np.ascontiguousarray(yp, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2:
        raise ValueError("X must be N x D")
    n, d = x.shape
    if yp.shape != (n * (n - 1) // 2,):
        raise ValueError(f"packed Y must have N(N-1)/2 = {n * (n - 1) // 2} entries, got {yp.shape}")
    return yp, x, n, d


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def keep_mask(n, heldout):
    """Training mask for a cross-validation fold (section 2.4): one byte per
    packed pair i < j, 0 for the held-out pairs (any order within a pair)."""
    keep = np.ones(n * (n - 1) // 2, dtype=np.uint8)
    for i, j in np.asarray(heldout, dtype=np.int64).reshape(-1, 2):
        a, b = (i, j) if i < j else (j, i)
        if a == b or a < 0 or b >= n:
            raise ValueError(f"bad held-out pair ({i}, {j})")
        keep[a * n - a * (a + 1) // 2 + (b - a - 1)] = 0
    return keep


def _keep_ptr(keep, n):
    if keep is None:
        return None, None
    k = np.ascontiguousarray(keep, dtype=np.uint8)
    if k.shape != (n * (n - 1) // 2,):
        raise ValueError("keep must hold one byte per packed pair")
    return k, _ptr(k)


def loglik(yp, x, sigma, nthreads=1, keep=None):
    """Return (L, sum_r): L = -M log sigma - sum_{i<j} r_ij (Eq. 2), over the
    pairs with keep != 0 when a training mask is given (M = their count)."""
    yp, x, n, d = _prep(yp, x)
    k, kp = _keep_ptr(keep, n)
    sr = np.zeros(1)
    ll = np.zeros(1)
    _check(_load().mdso_loglik_kept(n, d, _ptr(yp), kp, _ptr(x), float(sigma), int(nthreads), _ptr(sr),
                                    _ptr(ll)), "loglik")
    return float(ll[0]), float(sr[0])


def gradient(yp, x, sigma, rows=None, nthreads=1, with_abs=False, with_sq=False, keep=None):
    """Gradient of L in X (Eq. 9) for `rows` (all when None); optionally also
    S_ik = sum_j |term_ijk| (with_abs) and sqrt(sum_j term_ijk^2) (with_sq).
    keep: training mask (pairs with keep == 0 are left out)."""
    yp, x, n, d = _prep(yp, x)
    k, kp = _keep_ptr(keep, n)
    if rows is None:
        rr = None
        cnt = n
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int64)
        cnt = rr.shape[0]
    g = np.zeros((cnt, d))
    a = np.zeros((cnt, d)) if with_abs else None
    q = np.zeros((cnt, d)) if with_sq else None
    _check(_load().mdso_gradient_rows_kept(n, d, _ptr(yp), kp, _ptr(x), float(sigma),
                                           None if rr is None else _ptr(rr), cnt, int(nthreads), _ptr(g),
                                           None if a is None else _ptr(a), None if q is None else _ptr(q)),
           "gradient")
    out = (g,)
    if with_abs:
        out += (a,)
    if with_sq:
        out += (q,)
    return out if len(out) > 1 else g


def dsigma(yp, x, sigma, nthreads=1, keep=None):
    """d L / d sigma (Eq. 2 differentiated in sigma), over the kept pairs."""
    yp, x, n, d = _prep(yp, x)
    k, kp = _keep_ptr(keep, n)
    out = np.zeros(1)
    _check(_load().mdso_dsigma_kept(n, d, _ptr(yp), kp, _ptr(x), float(sigma), int(nthreads), _ptr(out)),
           "dsigma")
    return float(out[0])


def leapfrog(yp, x, p, sigma, eps, n_steps, w=1.0, lam=0.0, nthreads=1, keep=None):
    """n_steps leapfrog steps (M = I); returns (x, p, H0, H1)."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    p = np.array(p, dtype=np.float64, order="C", copy=True)
    n, d = x.shape
    k, kp = _keep_ptr(keep, n)
    if yp is None:
        ypp = None
    else:
        ypp = np.ascontiguousarray(yp, dtype=np.float32)
    h = np.zeros(2)
    _check(_load().mdso_leapfrog_kept(n, d, None if ypp is None else _ptr(ypp), kp, _ptr(x), _ptr(p),
                                      float(sigma), float(w), float(lam), float(eps), int(n_steps),
                                      int(nthreads), _ptr(h[0:]), h[1:].ctypes.data_as(_vp)), "leapfrog")
    return x, p, float(h[0]), float(h[1])


def hmc(yp, x, sigma, eps, n_steps, p_all, u_all, w=1.0, lam=0.0, nthreads=1, keep=None):
    """HMC with caller-supplied momenta (n_iter x N x D) and uniforms (n_iter);
    returns (x, accepted[n_iter], dH[n_iter])."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    n, d = x.shape
    k, kp = _keep_ptr(keep, n)
    p_all = np.ascontiguousarray(p_all, dtype=np.float64)
    u_all = np.ascontiguousarray(u_all, dtype=np.float64)
    n_iter = u_all.shape[0]
    if p_all.shape != (n_iter, n, d):
        raise ValueError("p_all must be n_iter x N x D")
    ypp = None if yp is None else np.ascontiguousarray(yp, dtype=np.float32)
    acc = np.zeros(n_iter, dtype=np.int32)
    dh = np.zeros(n_iter)
    _check(_load().mdso_hmc_kept(n, d, None if ypp is None else _ptr(ypp), kp, _ptr(x), float(sigma),
                                 float(w), float(lam), float(eps), int(n_steps), int(n_iter), _ptr(p_all),
                                 _ptr(u_all), int(nthreads), _ptr(acc), _ptr(dh)), "hmc")
    return x, acc.astype(bool), dh


def lpd(yp, heldout, xs, sigmas):
    """Log pointwise predictive density estimate (section 2.4) over the
    held-out pairs (K x 2) from S posterior draws: locations xs (S x N x D)
    and sigmas (S)."""
    yp = np.ascontiguousarray(yp, dtype=np.float32)
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    if xs.ndim == 2:
        xs = xs[None]
    S, n, d = xs.shape
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (S,)))
    pr = np.ascontiguousarray(heldout, dtype=np.int64).reshape(-1, 2)
    out = np.zeros(1)
    _check(_load().mdso_lpd(n, d, _ptr(yp), pr.shape[0], _ptr(pr), S, _ptr(xs), _ptr(sg), _ptr(out)), "lpd")
    return float(out[0])


def philox4x32_10(counter, key):
    """Philox4x32-10 block: 4 x uint32 counter, 2 x uint32 key -> 4 x uint32."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().mdso_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def draw_momentum(seed, chain, it, count):
    """Standard-normal momenta (count values) and the Metropolis uniform of
    HMC iteration `it` for chain `chain`, from the Philox stream keyed by the
    64-bit `seed`."""
    p = np.zeros(count)
    u = np.zeros(1)
    _load().mdso_draw_momentum(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, chain, it, count,
                               _ptr(p), _ptr(u))
    return p, float(u[0])


def sigma_mh(yp, x, sigma, step, shape, rate, z_all, u_all, w=1.0, keep=None, nthreads=1):
    """Random-walk Metropolis updates of log sigma given X with the prior
    sigma^-2 ~ Gamma(shape, rate) (w = 0: prior only).  Returns
    (sigma, accepted[n_iter])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    k, kp = _keep_ptr(keep, n)
    z = np.ascontiguousarray(z_all, dtype=np.float64)
    u = np.ascontiguousarray(u_all, dtype=np.float64)
    if z.shape != u.shape or z.ndim != 1:
        raise ValueError("z_all and u_all must be vectors of the same length")
    ypp = None if yp is None else np.ascontiguousarray(yp, dtype=np.float32)
    s = np.array([float(sigma)])
    acc = np.zeros(len(z), dtype=np.int32)
    _check(_load().mdso_sigma_mh(n, d, None if ypp is None else _ptr(ypp), kp, _ptr(x), _ptr(s), float(w), len(z),
                                 float(step), float(shape), float(rate), _ptr(z), _ptr(u), int(nthreads), _ptr(acc)),
           "sigma_mh")
    return float(s[0]), acc.astype(bool)


def sigma_draws(seed, chain, it):
    """(z, u) of sigma update `it` from the Philox stream keyed by `seed`."""
    z = np.zeros(1)
    u = np.zeros(1)
    _load().mdso_sigma_draws(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, chain, it, _ptr(z), _ptr(u))
    return float(z[0]), float(u[0])


def rwmh(yp, x, sigma, step, items, z_all, u_all, w=1.0, lam=0.0):
    """Single-item random-walk Metropolis (section 2.3's prior art):
    proposal t moves item items[t] by step * z_all[t]; accepted iff
    log u_t < log pi(X') - log pi(X).  Returns (x, accepted, dlogpi)."""
    x = np.array(x, dtype=np.float64, order="C")
    n, d = x.shape
    yp = np.ascontiguousarray(yp, dtype=np.float32) if w != 0.0 else np.zeros(1, dtype=np.float32)
    items = np.ascontiguousarray(items, dtype=np.int64)
    z = np.ascontiguousarray(z_all, dtype=np.float64).reshape(len(items), d)
    u = np.ascontiguousarray(u_all, dtype=np.float64)
    acc = np.zeros(len(items), dtype=np.int32)
    dl = np.zeros(len(items))
    _check(_load().mdso_rwmh(n, d, _ptr(yp), _ptr(x), sigma, w, lam, step, len(items), _ptr(items), _ptr(z),
                             _ptr(u), _ptr(acc), _ptr(dl)), "rwmh")
    return x, acc, dl


def rwmh_draws(seed, chain, it, n, d):
    """(item, z[D], u) of random-walk proposal `it` from Philox4x32-10
    (counters (it, 0, chain, 3) and (it, 1 + q, chain, 3))."""
    item = ctypes.c_int64()
    z = np.zeros(d)
    u = ctypes.c_double()
    _load().mdso_rwmh_draws(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, chain, it, n, d, ctypes.byref(item),
                            _ptr(z), ctypes.byref(u))
    return int(item.value), z, float(u.value)
