"""Shared helpers of the GPU parity tests (tolerances and comparisons).

Tolerances (stated for the hot path):
  log-likelihood: relative error <= 1e-6 (FP32C path), <= 1e-12 (FP64 path);
  gradient coordinates and dL/dsigma: relative error <= 1e-5 (FP32C),
  <= 1e-12 (FP64).
A relative error is ill-conditioned where a coordinate's terms cancel, so a
gradient coordinate also passes when
  (a) its condition number kappa = S / |g_ref| exceeds 1e3 (S = sum of the
      absolute values of its terms, from the oracle) and its absolute error
      is below max(tol * 1e-3, u) * S: terms summed in a precision of unit
      roundoff u can be off by u * S in the worst case (each term rounded
      once or twice on its way into a short partial sum), whatever the
      grouping of the sum (the strip length, chosen by timing, sets it);
      or
  (b) its absolute error is below 8 u * S2, S2 = sqrt(sum of its squared
      terms) and u the unit roundoff of the path (2^-24 for FP32C, 2^-53 for
      FP64): the size of the rounding error that any evaluation of the
      per-pair terms with a few units in the last place each leaves in their
      sum (random-walk model).
Coordinates that pass only through (a) or (b) are counted and reported, and
they must stay rare: at most ESCAPE_FRAC (0.1%) of the coordinates, and at
least one allowed on small cases (a regression that pushed many coordinates
into the escape branches fails even when each of them is within (a) or (b)).
"""
import numpy as np

TOL = {
    "fp32c": {"ll": 1e-6, "g": 1e-5, "u": 2.0 ** -24},
    "fp64": {"ll": 1e-12, "g": 1e-12, "u": 2.0 ** -53},
}
KAPPA = 1e3
ULPS = 8.0
ESCAPE_FRAC = 1e-3


def escape_cap(n):
    return max(1, int(ESCAPE_FRAC * n))


def grad_check(g, g_ref, s_abs, tol, what="gradient", s_sq=None, u=None):
    g = np.asarray(g, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    s_abs = np.asarray(s_abs, dtype=np.float64)
    err = np.abs(g - g_ref)
    rel_ok = err <= tol * np.abs(g_ref)
    kappa = s_abs / np.maximum(np.abs(g_ref), 1e-300)
    cond_ok = (kappa > KAPPA) & (err <= max(tol * 1e-3, u or 0.0) * s_abs)
    if s_sq is not None and u is not None:
        round_ok = err <= ULPS * u * np.asarray(s_sq, dtype=np.float64)
    else:
        round_ok = np.zeros_like(rel_ok)
    ok = rel_ok | cond_ok | round_ok
    rel = err / np.maximum(np.abs(g_ref), 1e-300)
    info = {
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "p999_rel": float(np.quantile(rel, 0.999)) if rel.size else 0.0,
        "n_kappa_branch": int(np.sum(~rel_ok & cond_ok)),
        "n_rounding_branch": int(np.sum(~rel_ok & ~cond_ok & round_ok)),
        "n": int(g.size),
    }
    bad = np.argwhere(~ok)
    assert bad.size == 0, (f"{what}: {len(bad)} of {g.size} coordinates out of tolerance {tol}; first "
                           f"{bad[:5].tolist()}: got {g[tuple(bad[0])]}, ref {g_ref[tuple(bad[0])]}, "
                           f"kappa {kappa[tuple(bad[0])]:.3g}; {info}")
    n_escape = info["n_kappa_branch"] + info["n_rounding_branch"]
    assert n_escape <= escape_cap(g.size), (f"{what}: {n_escape} of {g.size} coordinates passed only through "
                                            f"the cancellation or rounding branch (cap {escape_cap(g.size)}); {info}")
    return info


def scalar_check(v, ref, tol, scale=None, what="value"):
    err = abs(v - ref)
    lim = tol * abs(ref)
    if scale is not None and scale / max(abs(ref), 1e-300) > KAPPA:
        lim = max(lim, tol * 1e-3 * scale)
    assert err <= lim, f"{what}: got {v!r}, ref {ref!r}, rel err {err / max(abs(ref), 1e-300):.3e}, tol {tol}"
    return err / max(abs(ref), 1e-300)
