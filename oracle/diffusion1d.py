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


def implicit_T7_step(T, sig0, dx, dt, a=1.0, c=1.0, Cv=1.0, TL=None, TR=None, tol=1e-13, maxit=200, p=3.0):
    """One step of the fully implicit limit solver for sigma = sigma_0/T^3 (Sec. 6.5,
    Eq. diff_solver):

      (T^4 - T_n^4)/dt + (Cv/a)(T - T_n)/dt
          = 4c/(21 dx^2) [ k_{i+1/2} (T_{i+1}^7 - T_i^7) - k_{i-1/2} (T_i^7 - T_{i-1}^7) ],

    and for sigma_0/T^p (p given) the same with T^7 -> T^{p+4} and 21 -> 3 (p + 4): the
    limit flux a c T^p/(3 sigma_0) d(T^4)/dx = 4 a c/(3 (p + 4) sigma_0) d(T^{p+4})/dx.

    k_{i+1/2} = (1/sigma_0)_{i+1/2}, the mean of 1/sigma_0 of the two cells (the
    displayed average).  Walls (the paper does not print them): TL / TR given - the
    Dirichlet values T(0) = TL, T(L) = TR of the Marshak problem - enter through the
    half cell between the wall and the first cell centre, with k of that cell;
    None - zero flux.  Newton's method on the global system in the unknown u = T^4
    (its accumulation term keeps the Jacobian regular where the diffusion degenerates,
    T -> 0), tridiagonal Jacobian, iterates kept non-negative."""
    N = T.size
    Tn = np.asarray(T, dtype=np.float64)
    un = Tn ** 4
    inv = 1.0 / np.asarray(sig0, dtype=np.float64) * np.ones(N)
    kf = 0.5 * (inv[:-1] + inv[1:])                  # interior faces 1..N-1
    m = p + 4.0
    coef = 4.0 * c / (3.0 * m * dx ** 2)
    kL = 2.0 * inv[0] if TL is not None else 0.0     # half-cell distance at the walls
    kR = 2.0 * inv[-1] if TR is not None else 0.0
    bL = TL ** m if TL is not None else 0.0
    bR = TR ** m if TR is not None else 0.0
    u = un.copy()
    for _ in range(maxit):
        V = u ** (m / 4.0)                             # T^{p+4}
        flux = np.zeros(N)
        fi = kf * (V[1:] - V[:-1])
        flux[:-1] += fi
        flux[1:] -= fi
        flux[0] += kL * (bL - V[0])
        flux[-1] += kR * (bR - V[-1])
        F = (u - un) / dt + Cv / a * (u ** 0.25 - Tn) / dt - coef * flux
        dV = (m / 4.0) * u ** (m / 4.0 - 1.0)
        di = 1.0 / dt + Cv / a * 0.25 * np.maximum(u, 1e-300) ** -0.75 / dt
        di[:-1] += coef * kf * dV[:-1]
        di[1:] += coef * kf * dV[1:]
        di[0] += coef * kL * dV[0]
        di[-1] += coef * kR * dV[-1]
        ab = np.zeros((3, N))
        ab[0, 1:] = -coef * kf * dV[1:]
        ab[2, :-1] = -coef * kf * dV[:-1]
        ab[1] = di
        d = solve_banded((1, 1), ab, -F)
        unew = np.maximum(u + d, 0.0)
        step = np.max(np.abs(unew - u))
        u = unew
        if step <= tol * max(1.0, np.max(np.abs(u))):
            break
    return u ** 0.25


def front_position(T, dx, level=0.5):
    """x_f = the largest cell centre with T >= level (Sec. 6.5: where the wave stands);
    linear interpolation between that cell and the next."""
    i = np.nonzero(T >= level)[0]
    if i.size == 0:
        return 0.0
    j = i[-1]
    xc = (j + 0.5) * dx
    if j + 1 < T.size and T[j] != T[j + 1]:
        xc += dx * (T[j] - level) / (T[j] - T[j + 1])
    return xc
