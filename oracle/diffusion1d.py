"""Limit-equation solvers in 1D (oracle; test infrastructure only).

three_stage_step: the three-stage diffusion solver of Sec. 2, fully discrete
  (Eq. dis-diff for a T-independent sigma; the displayed fully discrete form after
  Eq. marshak-diff2 for sigma/T^3, reading the second node coefficient there as
  (T^{n+1*})^3 like the first).  Unknowns on cells; node coefficients
  (a c kappa/(3 sigma))_i with kappa = 1 or the node mean of T^3, and sigma_i the
  harmonic mean of the neighbouring cells.  Zero-flux walls (the even/odd scheme's
  reflecting wall has O = 0 there).
two_stage_step: the prediction/projection counter-example Eq. dis-diff-2.

The fully implicit reference solvers of Sec. 6 (Eq. imp_T and Eq. diff_solver) are
written with Newton's method on the global nonlinear system (tridiagonal Jacobian).
"""
import numpy as np
from scipy.linalg import solve_banded

from .scalar import quartic_root


def _node_harmonic(sig):
    l, r = sig[:-1], sig[1:]
    return 2.0 * l * r / (l + r)


def _diffusion_matrix(coef_node, dx, N):
    """Banded (ab, for solve_banded) form of -1/dx^2 [k_{j+1}(u_{j+1}-u_j) - k_j(u_j-u_{j-1})]
    with zero flux at the walls; coef_node has length N-1 (interior nodes 1..N-1)."""
    lo = np.zeros(N)
    up = np.zeros(N)
    lo[1:] = -coef_node / dx ** 2
    up[:-1] = -coef_node / dx ** 2
    di = -(lo + up)
    ab = np.zeros((3, N))
    ab[0, 1:] = up[:-1]
    ab[1] = di
    ab[2, :-1] = lo[1:]
    return ab, lo, di, up


def three_stage_step(T, sig, dx, dt, a=1.0, c=1.0, Cv=1.0, kind="const", Dd=3.0):
    """One step of the three-stage diffusion solver.  Returns (T_new, U_star)."""
    N = T.size
    U = T ** 4
    sn = _node_harmonic(sig)
    if kind == "const":
        kap_n = np.ones(N - 1)
    else:
        K = T ** 3
        kap_n = 0.5 * (K[:-1] + K[1:])
    # stage 1 (prediction): (U* - U)/dt = 4T^3/(4aT^3 + Cv) * div(ac kappa/(Dd sigma) grad U*)
    ab, lo, di, up = _diffusion_matrix(a * c * kap_n / (Dd * sn), dx, N)
    fac = 4.0 * T ** 3 / (4.0 * a * T ** 3 + Cv)
    ab1 = ab * 0.0
    ab1[0] = ab[0] * np.concatenate(([0.0], fac[:-1]))
    ab1[1] = 1.0 / dt + ab[1] * fac
    ab1[2] = ab[2] * np.concatenate((fac[1:], [0.0]))
    Ustar = solve_banded((1, 1), ab1, U / dt)
    # stage 2 (correction): a (T^4 - T^n^4)/dt + Cv (T - T^n)/dt = div(ac kappa*/(Dd sigma) grad U*)
    if kind == "const":
        kap2 = kap_n
    else:
        Ks = np.maximum(Ustar, 0.0) ** 0.75
        kap2 = 0.5 * (Ks[:-1] + Ks[1:])
    _, lo2, di2, up2 = _diffusion_matrix(a * c * kap2 / (Dd * sn), dx, N)
    flux = -(di2 * Ustar)
    flux[1:] -= lo2[1:] * Ustar[:-1]
    flux[:-1] -= up2[:-1] * Ustar[1:]
    A = a / dt * np.ones(N)
    B = Cv / dt * np.ones(N)
    R = a * U / dt + Cv * T / dt + flux
    Tn, _ = quartic_root(A, B, R)
    return Tn, Ustar


def two_stage_step(T, sig, dx, dt, a=1.0, c=1.0, Cv=1.0, Dd=3.0):
    """Eq. dis-diff-2: prediction then T = U^{1/4} (no correction)."""
    N = T.size
    U = T ** 4
    sn = _node_harmonic(sig)
    ab, lo, di, up = _diffusion_matrix(a * c / (Dd * sn), dx, N)
    fac = 4.0 * T ** 3 / (4.0 * a * T ** 3 + Cv)
    ab1 = np.zeros_like(ab)
    ab1[0] = ab[0] * np.concatenate(([0.0], fac[:-1]))
    ab1[1] = 1.0 / dt + ab[1] * fac
    ab1[2] = ab[2] * np.concatenate((fac[1:], [0.0]))
    Un = solve_banded((1, 1), ab1, U / dt)
    return np.maximum(Un, 0.0) ** 0.25


def implicit_T4_step(T, sig, dx, dt, a=1.0, c=1.0, Cv=1.0, Dd=3.0, tol=1e-14, maxit=100):
    """Eq. imp_T with every T^4 on the right at the new time level (the (T_i^n)^4 in
    the first flux difference is read as (T_i^{n+1})^4), sigma_{i+1/2} the harmonic
    node mean, zero-flux walls.  Newton on the global system."""
    N = T.size
    sn = _node_harmonic(sig)
    k = a * c / (Dd * sn) / dx ** 2
    x = T.copy()
    for _ in range(maxit):
        V = x ** 4
        F = a * (V - T ** 4) / dt + Cv * (x - T) / dt
        fl = np.zeros(N)
        fl[:-1] += k * (V[1:] - V[:-1])
        fl[1:] -= k * (V[1:] - V[:-1])
        F -= fl
        dV = 4.0 * x ** 3
        di = a * dV / dt + Cv / dt
        di[:-1] += k * dV[:-1]
        di[1:] += k * dV[1:]
        ab = np.zeros((3, N))
        ab[0, 1:] = -k * dV[1:]
        ab[2, :-1] = -k * dV[:-1]
        ab[1] = di
        dx_ = solve_banded((1, 1), ab, -F)
        x = np.maximum(x + dx_, 0.0)
        if np.max(np.abs(dx_)) <= tol * max(1.0, np.max(np.abs(x))):
            break
    return x
