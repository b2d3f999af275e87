"""Shared helpers of the GPU parity tests (tolerances and comparisons).

Tolerances (stated for the hot path):
  log-likelihood: relative error <= 1e-6 (FP32C path), <= 1e-12 (FP64 path);
  gradient coordinates and dL/dsigma: relative error <= 1e-5 (FP32C),
  <= 1e-12 (FP64).
A relative error is ill-conditioned where a coordinate's terms cancel, so a
gradient coordinate also passes when
  (a) its condition number kappa = S / |g_ref| exceeds 1e3 (S = sum of the
      absolute values of its terms, from the oracle), or it lies below the
      escape line defined next, and its absolute error is below
      max(tol * 1e-3, u) * S: terms summed in a precision of unit roundoff u
      can be off by u * S in the worst case (each term rounded once or twice
      on its way into a short partial sum), whatever the grouping of the sum
      (the pass shape, chosen by timing, sets it); or
  (b) its absolute error is below 8 u * S2, S2 = sqrt(sum of its squared
      terms) and u the unit roundoff of the path (2^-24 for FP32C, 2^-53 for
      FP64): the size of the rounding error that any evaluation of the
      per-pair terms with a few units in the last place each leaves in their
      sum (random-walk model).
Coordinates that pass only through (a) or (b) are counted and reported, and
only ill-conditioned coordinates may use them: each must have
|g_ref| <= ESCAPE_SLACK * ULPS * u / tol * S2, the size below which even an
evaluation with a few units in the last place per term cannot promise the
relative tolerance (8 u S2 >= tol |g_ref|), with a factor 2 of slack.  A
coordinate above that line that misses the relative tolerance fails, so a
regression that pushes well-conditioned coordinates into the escape branches
is caught (how many coordinates sit below the line depends on the data: a
handful per thousand in six dimensions at N = 333, none at most sizes).
"""
import json
import os

import numpy as np


def _log(kind, what, info):
    """Append one record to the JSON-lines file named by MDS_PARITY_LOG (the
    observed errors of every check, for the record of stated errors)."""
    path = os.environ.get("MDS_PARITY_LOG")
    if not path:
        return
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "kind": kind, "what": what}
    rec.update(info)
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")

TOL = {
    "fp32c": {"ll": 1e-6, "g": 1e-5, "u": 2.0 ** -24},
    "fp64": {"ll": 1e-12, "g": 1e-12, "u": 2.0 ** -53},
}
KAPPA = 1e3
ULPS = 8.0
ESCAPE_SLACK = 2.0


def grad_check(g, g_ref, s_abs, tol, what="gradient", s_sq=None, u=None):
    g = np.asarray(g, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    s_abs = np.asarray(s_abs, dtype=np.float64)
    err = np.abs(g - g_ref)
    rel_ok = err <= tol * np.abs(g_ref)
    kappa = s_abs / np.maximum(np.abs(g_ref), 1e-300)
    # the cancellation branch: kappa above KAPPA, or (with S2 known) the
    # coordinate below the escape line, where even a few ulps per term cannot
    # promise the relative tolerance and the FP32 sums' own rounding, up to
    # u S, decides
    ill = kappa > KAPPA
    if s_sq is not None and u is not None:
        ill = ill | (np.abs(g_ref) <= ESCAPE_SLACK * ULPS * u / tol * np.asarray(s_sq, dtype=np.float64))
    cond_ok = ill & (err <= max(tol * 1e-3, u or 0.0) * s_abs)
    if s_sq is not None and u is not None:
        round_ok = err <= ULPS * u * np.asarray(s_sq, dtype=np.float64)
    else:
        round_ok = np.zeros_like(rel_ok)
    ok = rel_ok | cond_ok | round_ok
    rel = err / np.maximum(np.abs(g_ref), 1e-300)
    escape = ~rel_ok & (cond_ok | round_ok)
    info = {
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "p999_rel": float(np.quantile(rel, 0.999)) if rel.size else 0.0,
        "max_rel_well_conditioned": float(rel[~escape].max()) if np.any(~escape) else 0.0,
        "n_kappa_branch": int(np.sum(~rel_ok & cond_ok)),
        "n_rounding_branch": int(np.sum(~rel_ok & ~cond_ok & round_ok)),
        "n": int(g.size),
    }
    if s_sq is not None and u is not None:
        ratio = np.abs(g_ref) / np.maximum(np.asarray(s_sq, dtype=np.float64), 1e-300)
        info["escape_max_g_over_s2"] = float(ratio[escape].max()) if np.any(escape) else 0.0
    _log("grad", what, dict(info, tol=tol, n_bad=int(np.sum(~ok))))
    bad = np.argwhere(~ok)
    assert bad.size == 0, (f"{what}: {len(bad)} of {g.size} coordinates out of tolerance {tol}; first "
                           f"{bad[:5].tolist()}: got {g[tuple(bad[0])]}, ref {g_ref[tuple(bad[0])]}, "
                           f"kappa {kappa[tuple(bad[0])]:.3g}; {info}")
    if s_sq is not None and u is not None:
        line = ESCAPE_SLACK * ULPS * u / tol
        info["escape_line"] = line
        bad_esc = np.argwhere(escape & (ratio > line))
        assert bad_esc.size == 0, (f"{what}: {len(bad_esc)} well-conditioned coordinates (|g| > {line:.3g} S2) "
                                   f"passed only through the cancellation or rounding branch; first "
                                   f"{bad_esc[:5].tolist()}; {info}")
    return info


def scalar_check(v, ref, tol, scale=None, what="value", abs_floor=0.0):
    """|v - ref| <= tol |ref|, or tol * 1e-3 * scale where scale / |ref| >
    KAPPA (cancelling terms), or abs_floor (an absolute error bound of the
    path's arithmetic that the caller states)."""
    err = abs(v - ref)
    lim = tol * abs(ref)
    if scale is not None and scale / max(abs(ref), 1e-300) > KAPPA:
        lim = max(lim, tol * 1e-3 * scale)
    lim = max(lim, abs_floor)
    _log("scalar", what, {"rel": err / max(abs(ref), 1e-300), "tol": tol, "lim_rel": lim / max(abs(ref), 1e-300)})
    assert err <= lim, f"{what}: got {v!r}, ref {ref!r}, rel err {err / max(abs(ref), 1e-300):.3e}, tol {tol}"
    return err / max(abs(ref), 1e-300)
