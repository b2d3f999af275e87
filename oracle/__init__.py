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
            lib.mdso_loglik.argtypes = [_i64, _int, _vp, _vp, _dbl, _int, _vp, _vp]
            lib.mdso_gradient_rows.argtypes = [_i64, _int, _vp, _vp, _dbl, _vp, _i64, _int, _vp, _vp, _vp]
            lib.mdso_dsigma.argtypes = [_i64, _int, _vp, _vp, _dbl, _int, _vp]
            lib.mdso_leapfrog.argtypes = [_i64, _int, _vp, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int,
                                          _int, _vp, _vp]
            lib.mdso_hmc.argtypes = [_i64, _int, _vp, _vp, _dbl, _dbl, _dbl, _dbl, _int, _int, _vp,
                                     _vp, _int, _vp, _vp]
            lib.mdso_philox4x32_10.argtypes = [_vp, _vp, _vp]
            lib.mdso_draw_momentum.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, _i64, _vp, _vp]
            for f in ("mdso_loglik", "mdso_gradient_rows", "mdso_dsigma", "mdso_leapfrog",
                      "mdso_hmc"):
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


def loglik(yp, x, sigma, nthreads=1):
    """Return (L, sum_r): L = -M log sigma - sum_{i<j} r_ij (Eq. 2)."""
    yp, x, n, d = _prep(yp, x)
    sr = np.zeros(1)
    ll = np.zeros(1)
    _check(_load().mdso_loglik(n, d, _ptr(yp), _ptr(x), float(sigma), int(nthreads), _ptr(sr),
                               _ptr(ll)), "loglik")
    return float(ll[0]), float(sr[0])


def gradient(yp, x, sigma, rows=None, nthreads=1, with_abs=False, with_sq=False):
    """Gradient of L in X (Eq. 9) for `rows` (all when None); optionally also
    S_ik = sum_j |term_ijk| (with_abs) and sqrt(sum_j term_ijk^2) (with_sq)."""
    yp, x, n, d = _prep(yp, x)
    if rows is None:
        rr = None
        cnt = n
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int64)
        cnt = rr.shape[0]
    g = np.zeros((cnt, d))
    a = np.zeros((cnt, d)) if with_abs else None
    q = np.zeros((cnt, d)) if with_sq else None
    _check(_load().mdso_gradient_rows(n, d, _ptr(yp), _ptr(x), float(sigma),
                                      None if rr is None else _ptr(rr), cnt, int(nthreads), _ptr(g),
                                      None if a is None else _ptr(a), None if q is None else _ptr(q)), "gradient")
    out = (g,)
    if with_abs:
        out += (a,)
    if with_sq:
        out += (q,)
    return out if len(out) > 1 else g


def dsigma(yp, x, sigma, nthreads=1):
    """d L / d sigma (Eq. 2 differentiated in sigma)."""
    yp, x, n, d = _prep(yp, x)
    out = np.zeros(1)
    _check(_load().mdso_dsigma(n, d, _ptr(yp), _ptr(x), float(sigma), int(nthreads), _ptr(out)),
           "dsigma")
    return float(out[0])


def leapfrog(yp, x, p, sigma, eps, n_steps, w=1.0, lam=0.0, nthreads=1):
    """n_steps leapfrog steps (M = I); returns (x, p, H0, H1)."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    p = np.array(p, dtype=np.float64, order="C", copy=True)
    n, d = x.shape
    if yp is None:
        ypp = None
    else:
        ypp = np.ascontiguousarray(yp, dtype=np.float32)
    h = np.zeros(2)
    _check(_load().mdso_leapfrog(n, d, None if ypp is None else _ptr(ypp), _ptr(x), _ptr(p),
                                 float(sigma), float(w), float(lam), float(eps), int(n_steps),
                                 int(nthreads), _ptr(h[0:]), h[1:].ctypes.data_as(_vp)), "leapfrog")
    return x, p, float(h[0]), float(h[1])


def hmc(yp, x, sigma, eps, n_steps, p_all, u_all, w=1.0, lam=0.0, nthreads=1):
    """HMC with caller-supplied momenta (n_iter x N x D) and uniforms (n_iter);
    returns (x, accepted[n_iter], dH[n_iter])."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    n, d = x.shape
    p_all = np.ascontiguousarray(p_all, dtype=np.float64)
    u_all = np.ascontiguousarray(u_all, dtype=np.float64)
    n_iter = u_all.shape[0]
    if p_all.shape != (n_iter, n, d):
        raise ValueError("p_all must be n_iter x N x D")
    ypp = None if yp is None else np.ascontiguousarray(yp, dtype=np.float32)
    acc = np.zeros(n_iter, dtype=np.int32)
    dh = np.zeros(n_iter)
    _check(_load().mdso_hmc(n, d, None if ypp is None else _ptr(ypp), _ptr(x), float(sigma),
                            float(w), float(lam), float(eps), int(n_steps), int(n_iter), _ptr(p_all),
                            _ptr(u_all), int(nthreads), _ptr(acc), _ptr(dh)), "hmc")
    return x, acc.astype(bool), dh


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
