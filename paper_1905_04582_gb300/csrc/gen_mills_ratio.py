"""Fit the rational approximation of the normal Mills ratio used by the FP32
pair kernel and write ``mills_ratio_coeffs.h``.

The FP32 kernel needs Phi(z) = 1 - Q(z) for z = delta / sigma >= 0, where
Q(z) = phi(z) R(z) and R is the Mills ratio.  Since the kernel already has
phi(z) (one exp2), it approximates R(z) by a rational function
P(z) / D(z), deg P = deg D = 3, D(0) = 1, fitted so that the *absolute* error
in Q, max_z phi(z) |R(z) - P(z)/D(z)|, is minimal over z in [0, 14] (beyond
14, phi(z) < 1e-42 underflows FP32 and Q is 0).  The weight phi(z) is what
makes a degree-(3,3) rational enough: Phi's FP32 spacing near 1 is 6e-8,
while the fit error is below 1e-8.

Method: the linearised weighted least-squares problem
phi (R D - P) = 0 is solved, then re-weighted by 1/|D| (Loeb's iteration)
and by Lawson's multiplicative weight update towards the minimax solution.
Reference values of Q come from mpmath's normal CDF at 30 digits.

Run:  python gen_mills_ratio.py  (needs numpy and mpmath; the header is
committed, the build does not run this script).
"""
import os

import mpmath
import numpy as np

P_DEG, D_DEG = 3, 3
Z_MAX = 14.0


def _reference():
    mpmath.mp.dps = 30
    z = np.concatenate([np.linspace(0.0, 8.0, 8001), np.linspace(8.0, Z_MAX, 1201)[1:]])
    phi = np.array([float(mpmath.npdf(v)) for v in z])
    q = np.array([float(mpmath.ncdf(-v)) for v in z])
    return z, phi, q / phi


def _eval(c, z):
    p = np.polyval(c[:P_DEG + 1][::-1], z)
    d = np.polyval(np.concatenate([[1.0], c[P_DEG + 1:]])[::-1], z)
    return p, d


def fit():
    z, phi, r = _reference()
    cols = [-phi * z ** k for k in range(P_DEG + 1)] + [phi * r * z ** k for k in range(1, D_DEG + 1)]
    a = np.array(cols).T
    b = -phi * r
    c, *_ = np.linalg.lstsq(a, b, rcond=None)
    for _ in range(30):  # Loeb: divide out the current denominator
        _, d = _eval(c, z)
        w = 1.0 / np.abs(d)
        c, *_ = np.linalg.lstsq(a * w[:, None], b * w, rcond=None)
    lw = np.ones_like(z)
    best = None
    for _ in range(400):  # Lawson: push towards equal-ripple error
        p, d = _eval(c, z)
        err = phi * (r - p / d)
        e = np.abs(err).max()
        if best is None or e < best[0]:
            best = (e, c.copy())
        lw = lw * (np.abs(err) / e + 1e-3) ** 0.5
        lw /= lw.max()
        w = lw / np.abs(d)
        c, *_ = np.linalg.lstsq(a * w[:, None], b * w, rcond=None)
    e, c = best
    zz = np.logspace(-3, 12, 4000)
    _, dd = _eval(c, zz)
    assert (dd > 0).all(), "denominator must stay positive on z >= 0"
    return e, c


def main():
    e, c = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_mills_ratio.py -- do not edit.",
        "// Normal Mills ratio R(z) = Q(z) / phi(z) ~= P(z) / D(z) on z >= 0, with",
        "// P(z) = p0 + p1 z + p2 z^2 + p3 z^3 and D(z) = 1 + d1 z + d2 z^2 + d3 z^3,",
        f"// fitted for minimal absolute error in Q = phi R: max |dQ| = {e:.3e} on [0, {Z_MAX:g}].",
        "#pragma once",
        f"static const double kMillsP[{P_DEG + 1}] = {{" + ", ".join(f"{v:.17e}" for v in c[:P_DEG + 1]) + "};",
        f"static const double kMillsD[{D_DEG + 1}] = {{1.0, " + ", ".join(f"{v:.17e}" for v in c[P_DEG + 1:]) + "};",
        f"static const double kMillsMaxAbsErrQ = {e:.3e};",
        "",
    ]
    with open(os.path.join(here, "mills_ratio_coeffs.h"), "w") as f:
        f.write("\n".join(lines))
    print("max |dQ| =", e)


if __name__ == "__main__":
    main()
