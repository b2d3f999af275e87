"""Shared helpers of the GPU parity tests (tolerances and comparisons).

Tolerances (stated for the hot path):
  log-likelihood: relative error <= 1e-6 (FP32C path), <= 1e-12 (FP64 path);
  gradient coordinates and dL/dsigma: relative error <= 1e-5 (FP32C),
  <= 1e-12 (FP64).
Near cancellation a relative error is ill-conditioned, so a coordinate whose
condition number kappa = S / |g_ref| exceeds 1e3 (S = sum of the absolute
values of its terms, returned by the oracle) passes when its absolute error
is below tol * 1e-3 * S instead; such coordinates are counted and printed.
"""
import numpy as np

TOL = {
    "fp32c": {"ll": 1e-6, "g": 1e-5},
    "fp64": {"ll": 1e-12, "g": 1e-12},
}
KAPPA = 1e3


def grad_check(g, g_ref, s_abs, tol, what="gradient"):
    g = np.asarray(g, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    s_abs = np.asarray(s_abs, dtype=np.float64)
    err = np.abs(g - g_ref)
    rel_ok = err <= tol * np.abs(g_ref)
    kappa = s_abs / np.maximum(np.abs(g_ref), 1e-300)
    cond_ok = (kappa > KAPPA) & (err <= tol * 1e-3 * s_abs)
    ok = rel_ok | cond_ok
    n_cond = int(np.sum(~rel_ok & cond_ok))
    rel = err / np.maximum(np.abs(g_ref), 1e-300)
    info = {
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "p999_rel": float(np.quantile(rel, 0.999)) if rel.size else 0.0,
        "n_kappa_branch": n_cond,
        "n": int(g.size),
    }
    bad = np.argwhere(~ok)
    assert bad.size == 0, (f"{what}: {len(bad)} of {g.size} coordinates out of tolerance {tol}; first "
                           f"{bad[:5].tolist()}: got {g[tuple(bad[0])]}, ref {g_ref[tuple(bad[0])]}, "
                           f"kappa {kappa[tuple(bad[0])]:.3g}; {info}")
    return info


def scalar_check(v, ref, tol, scale=None, what="value"):
    err = abs(v - ref)
    lim = tol * abs(ref)
    if scale is not None and scale / max(abs(ref), 1e-300) > KAPPA:
        lim = max(lim, tol * 1e-3 * scale)
    assert err <= lim, f"{what}: got {v!r}, ref {ref!r}, rel err {err / max(abs(ref), 1e-300):.3e}, tol {tol}"
    return err / max(abs(ref), 1e-300)
