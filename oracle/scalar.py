"""Per-cell scalar nonlinear solve of the correction step (oracle; test infrastructure only).

Eq. Tnp1 (Sec. 4, correction step) and its sigma/T^3 form (Sec. 5, sum of
Eq. dis-cor-marshak4 and Eq. dis-cor-marshak5) reduce, in every cell, to

    A T^4 + B T = R,    A >= 0, B >= 0,

with A, B, R defined in grte1d.correction_temperature.  For T >= 0 the left side
is convex and increasing, so for R > 0 there is exactly one non-negative root and
it lies in (0, T_hi] with T_hi = min((R/A)^(1/4), R/B).  Newton's method started at
T_hi decreases monotonically to that root (convexity), so the iteration below is
run until the iterate stops decreasing, i.e. until it has converged to rounding.
The paper only asks for "standard iterative solvers such as Newton's method"
(remark after Eq. dis-diff).
"""
import numpy as np


def quartic_root(A, B, R, max_iter=200):
    """Non-negative root of A T^4 + B T = R, elementwise over arrays.

    R <= 0 gives T = 0 (no positive root); A = B = 0 gives NaN (undetermined) and
    the caller decides.  Returns (T, iterations) with iterations per element.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    A, B, R = np.broadcast_arrays(A, B, R)
    T = np.zeros(R.shape)
    its = np.zeros(R.shape, dtype=np.int64)
    for idx in np.ndindex(R.shape):
        a, b, r = float(A[idx]), float(B[idx]), float(R[idx])
        if a == 0.0 and b == 0.0:
            T[idx] = np.nan
            continue
        if r <= 0.0:
            T[idx] = 0.0
            continue
        hi = np.inf
        if a > 0.0:
            hi = (r / a) ** 0.25
        if b > 0.0:
            hi = min(hi, r / b)
        t = hi
        n = 0
        while n < max_iter:
            f = a * t ** 4 + b * t - r
            fp = 4.0 * a * t ** 3 + b
            t_new = t - f / fp
            n += 1
            if not (t_new < t):
                break
            t = t_new
        T[idx] = t
        its[idx] = n
    return T, its
