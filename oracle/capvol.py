"""Hyperspherical-cap volume fraction (oracle; test infrastructure only).

Sec. 5, "Intersection Volume Approximation": partition P_i is approximated by
the half-space beyond the perpendicular bisector of c_0 and c_i.  The part of
the ball B(q, rho) inside that half-space is a cap whose height is h = rho - t,
t being the distance from q to the bisector.  By Li (2010), in d dimensions the
cap holds the fraction

    u(t, rho) = 1/2 * I_x((d + 1) / 2, 1 / 2),   x = (2 rho h - h^2) / rho^2 = 1 - (t / rho)^2

of the ball for 0 <= t < rho, and 0 for t >= rho.  I_x(a, b) is the
regularised incomplete beta function; scipy's `betainc` evaluates it here (a
library routine used as one step).

Sec. 5, "Performance Optimizations": I_x is tabulated at 1024 evenly spaced
points of [0, 1] and interpolated linearly.  Reading: the points are
x_j = j / 1023 for j = 0..1023, so both ends are included.
"""

import numpy as np
from scipy.special import betainc

TABLE_POINTS = 1024


def beta_shape(d):
    """(a, b) of the incomplete beta function for dimension d."""
    return 0.5 * (d + 1), 0.5


def cap_fraction(t, rho, d):
    """Exact cap fraction u(t, rho) for arrays t (>= 0) and a scalar rho."""
    t = np.asarray(t, dtype=np.float64)
    u = np.zeros_like(t)
    if not (rho > 0.0):
        return u
    inside = t < rho
    s = t[inside] / rho
    x = 1.0 - s * s
    a, b = beta_shape(d)
    u[inside] = 0.5 * betainc(a, b, x)
    return u


def beta_table(d):
    """I_x((d+1)/2, 1/2) at x_j = j / 1023, j = 0..1023."""
    a, b = beta_shape(d)
    xs = np.arange(TABLE_POINTS, dtype=np.float64) / (TABLE_POINTS - 1)
    return betainc(a, b, xs)


def interp_table(table, x):
    """Linear interpolation of the tabulated I_x at x in [0, 1]."""
    x = np.asarray(x, dtype=np.float64)
    f = x * (TABLE_POINTS - 1)
    j = np.floor(f).astype(np.int64)
    j = np.clip(j, 0, TABLE_POINTS - 2)
    w = f - j
    return table[j] + w * (table[j + 1] - table[j])


def cap_fraction_table(t, rho, table):
    """Cap fraction with I_x taken from the 1024-point table."""
    t = np.asarray(t, dtype=np.float64)
    u = np.zeros_like(t)
    if not (rho > 0.0):
        return u
    inside = t < rho
    s = t[inside] / rho
    u[inside] = 0.5 * interp_table(table, 1.0 - s * s)
    return u
