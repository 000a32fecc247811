"""OSPA distance between a set of estimated and a set of true points (evaluation metric).

Schuhmacher, Vo and Vo (2008): for X with m points and Y with n points, m <= n,
    d_p^(c)(X, Y) = ( (1/n) [ min_pi sum_{i=1..m} d^(c)(x_i, y_pi(i))^p + c^p (n - m) ] )^(1/p),
with d^(c)(x, y) = min(c, |x - y|) and the minimum over the injections pi of X into Y;
d = 0 when both sets are empty and c when exactly one is.  The assignment is solved as
a linear assignment on the cut-off distances raised to p (scipy's Hungarian-type
solver).  The filter's map is scored as the OSPA between the SFV estimates of the
declared PFs and the true SFVs (c and p stated by the caller).
"""
from __future__ import annotations

import numpy as np


def ospa(X: np.ndarray, Y: np.ndarray, c: float, p: float = 2.0) -> float:
    """OSPA distance of point sets X (m x d) and Y (n x d), both 2-D arrays (m or n may be
    0), with cut-off c and order p."""
    from scipy.optimize import linear_sum_assignment
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    m, n = len(X), len(Y)
    if m == 0 and n == 0:
        return 0.0
    if m == 0 or n == 0:
        return float(c)
    if m > n:
        X, Y, m, n = Y, X, n, m
    D = np.minimum(np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=-1), c) ** p
    r, k = linear_sum_assignment(D)
    return float(((D[r, k].sum() + c ** p * (n - m)) / n) ** (1.0 / p))
