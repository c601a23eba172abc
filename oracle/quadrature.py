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


def level_symmetric_s8():
    """Level-symmetric S8 set on the unit sphere (80 directions), one construction of
    the standard family (the paper prescribes none; reading Q16).

    Direction cosines take the four levels mu_i^2 = (1 + 6 (i-1))/21, i = 1..4 (so
    mu_1^2 = 1/21 and each step adds 2 (1 - 3 mu_1^2)/(N - 2) with N = 8).  In one
    octant the directions are (mu_a, mu_b, mu_c) with a + b + c = 6: the permutations
    of (1,1,4), (1,2,3) and (2,2,2), ten directions in three weight classes.  The
    three class weights are fixed by even moment conditions of the full sphere:
    sum w = 1, sum w mu_x^4 = 1/5 and sum w mu_x^6 = 1/7 (sum w mu_x^2 = 1/3 is
    not a fourth condition: it follows from sum w = 1, mu_x^2 + mu_y^2 + mu_z^2 = 1
    and the octant symmetry).

    Returns (dirs, w): dirs (80, 3), w (80,), sum(w) = 1.
    """
    m = np.array([(1.0 + 6.0 * i) / 21.0 for i in range(4)])    # mu_i^2, i = 0..3
    mu = np.sqrt(m)
    classes = {(0, 0, 3): 0, (0, 1, 2): 1, (1, 1, 1): 2}
    octant = []
    for a in range(4):
        for b in range(4):
            for c_ in range(4):
                if a + b + c_ == 3:      # 0-based levels summing to 6 - 3
                    octant.append((a, b, c_, classes[tuple(sorted((a, b, c_)))]))
    # moment equations over the full sphere (8 octants, per weight class)
    M = np.zeros((3, 3))
    rhs = np.array([1.0, 1.0 / 5.0, 1.0 / 7.0])
    for a, b, c_, cl in octant:
        M[0, cl] += 8.0
        M[1, cl] += 8.0 * m[a] ** 2
        M[2, cl] += 8.0 * m[a] ** 3
    wc = np.linalg.solve(M, rhs)
    dirs, w = [], []
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for sz in (1.0, -1.0):
                for a, b, c_, cl in octant:
                    dirs.append((sx * mu[a], sy * mu[b], sz * mu[c_]))
                    w.append(wc[cl])
    return np.array(dirs), np.array(w)


def s8_pairs_2d():
    """The 2D even/odd pair set from S8 (reading Q16): the 40 directions with a
    positive third cosine, projected on the (x, y) plane, each weight doubled; the
    directions come in pairs Omega, -Omega in the plane.  Each pair is represented
    by its member with mu > 0; the pair weight is the sum of the two members'
    weights, so the 20 pair weights sum to 1.

    Returns (mu, eta, w), each (20,), ordered by (mu, eta).
    """
    dirs, w = level_symmetric_s8()
    up = dirs[:, 2] > 0
    d, ww = dirs[up, :2], 2.0 * w[up]
    rep = d[:, 0] > 0
    mu, eta, wp = d[rep, 0], d[rep, 1], ww[rep]
    # the partner (-mu, -eta) of each representative carries the same weight (the
    # set is symmetric under inversion in the plane)
    wp = 2.0 * wp
    wp = wp / np.sum(wp)
    order = np.lexsort((eta, mu))
    return mu[order], eta[order], wp[order]
