"""Angular quadratures for the velocity variable (oracle; test infrastructure only).

Sec. 4 writes the 1D angular average as <f> = (1/2) int_{-1}^{1} f dv and, for the
even/odd parity unknowns, integrals over v in (0, 1) (Eq. dis-pre3, Eq. Tnp1).  The
paper leaves the velocity grid open ("we do not delineate on velocity
discretization", remark after Eq. dis-pre); the workloads use Gauss-Legendre.

gauss_legendre_half(n_v): the n_v-point Gauss-Legendre rule on [-1, 1] (numpy's
routine), keeping the n_v/2 positive nodes.  For an even integrand
int_0^1 f dv = (1/2) sum_all W f = sum_{v>0} W f, so the positive-node weights are
used unchanged and they sum to 1 = int_0^1 dv.
"""
import numpy as np


def gauss_legendre_half(n_v):
    """Return (v, w): the n_v/2 positive Gauss-Legendre nodes in increasing order and
    their weights, normalised so that sum(w) = int_0^1 dv = 1."""
    if n_v < 2 or n_v % 2:
        raise ValueError("n_v must be a positive even number")
    x, W = np.polynomial.legendre.leggauss(n_v)
    pos = x > 0
    v = x[pos]
    w = W[pos]
    order = np.argsort(v)
    return v[order].astype(np.float64), w[order].astype(np.float64)
