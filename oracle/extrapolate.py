"""Extrapolation of a DDA result to zero dipole size (Sec. 3.2).

Test infrastructure only (see oracle/__init__.py).

The paper runs the same problem at several discretisations and fits the
dependence of the result on the dipole size d with a quadratic function,
assuming the error of each point scales as d^3, then doubles the standard
error of the value at d = 0 for a nominal 95 % confidence interval.

Reading (the paper gives no formulas): the quadratic is the full
a0 + a1 d + a2 d^2; "errors scale as d^3" means standard deviations
sigma_i = s d_i^3 with one unknown scale s, so the fit is weighted least
squares with weights d_i^-6 and s^2 estimated from the weighted residuals
(chi^2 / (n - 3)); the standard error of a0 is the square root of the (0, 0)
element of s^2 (X^T W X)^-1.  The normal equations are written out here.
"""
from __future__ import annotations

import numpy as np


def extrapolate_to_zero(d, values):
    """Return (value at d = 0, half-width of the 95 % interval) for n >= 4
    points (d_i > 0); with exactly 3 points the fit interpolates and the
    interval is reported as 0."""
    d = np.asarray(d, dtype=np.float64)
    y = np.asarray(values, dtype=np.float64)
    n = len(d)
    if n < 3 or np.any(d <= 0):
        raise ValueError("need at least 3 positive dipole sizes")
    X = np.stack([np.ones(n), d, d * d], axis=1)
    w = d ** -6.0
    XtWX = X.T @ (w[:, None] * X)
    XtWy = X.T @ (w * y)
    a = np.linalg.solve(XtWX, XtWy)
    if n == 3:
        return float(a[0]), 0.0
    r = y - X @ a
    s2 = float(np.sum(w * r * r) / (n - 3))
    cov = s2 * np.linalg.inv(XtWX)
    return float(a[0]), float(2.0 * np.sqrt(cov[0, 0]))
