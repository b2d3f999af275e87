// Generated by gen_mills_ratio.py -- do not edit.
// Normal Mills ratio R(z) = Q(z) / phi(z) ~= P(z) / D(z) on z >= 0, with
// P(z) = p0 + p1 z + p2 z^2 + p3 z^3 and D(z) = 1 + d1 z + d2 z^2 + d3 z^3,
// fitted for minimal absolute error in Q = phi R: max |dQ| = 9.444e-09 on [0, 14].
#pragma once
static const double kMillsP[4] = {1.25331416095758663e+00, 4.62400036964757288e-01, 8.70669450201149997e-02, -3.69359157179304821e-04};
static const double kMillsD[4] = {1.0, 1.16682798810314714e+00, 5.00442683968438606e-01, 8.16509734108939733e-02};
static const double kMillsMaxAbsErrQ = 9.444e-09;
