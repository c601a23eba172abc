"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of these compares the oracle with
itself: the references are closed forms, high-precision solutions, invariants of
the discrete scheme, and separately written limit solvers.
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import grte1d as g
from oracle import diffusion1d as dif
from oracle.quadrature import gauss_legendre_half
from oracle.scalar import quartic_root


def _problem(N=12, nv=8, eps=1e-2, kind="t3", sig=1.0, bc="inflow", bL=1.0, bR=0.0, cfl=0.5):
    v, w = gauss_legendre_half(nv)
    return g.Problem(N=N, v=v, w=w, sig=sig, eps=eps, dt=cfl / N, kind=kind, bc=bc,
                     bL=np.full(v.size, bL), bR=np.full(v.size, bR))


def _bumpy_T(N, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(N) + 0.5) / N
    return 0.1 * np.exp(0.3 * rng.standard_normal(N)) + 0.5 * np.exp(-40 * (x - 0.5) ** 2)


# ---------------------------------------------------------------- quadrature (Sec. 4)
@pytest.mark.parametrize("nv", [2, 8, 16, 64])
def test_gauss_legendre_half_moments(nv):
    """<1> = 1, <v^2> = 1/3, <v^4> = 1/5 over v in (0,1): exact for Gauss-Legendre."""
    v, w = gauss_legendre_half(nv)
    assert v.size == nv // 2 and np.all(v > 0) and np.all(np.diff(v) > 0)
    assert abs(w.sum() - 1.0) < 1e-14
    assert abs(np.sum(w * v ** 2) - 1.0 / 3.0) < 1e-14
    if nv >= 4:
        assert abs(np.sum(w * v ** 4) - 0.2) < 1e-14


# ---------------------------------------------------------------- scalar solve (Eq. Tnp1)
def test_quartic_root_vs_high_precision_bisection():
    rng = np.random.default_rng(5)
    A = 10.0 ** rng.uniform(-6, 6, 200)
    B = 10.0 ** rng.uniform(-6, 6, 200)
    R = 10.0 ** rng.uniform(-8, 8, 200)
    T, its = quartic_root(A, B, R)
    mp.mp.dps = 40
    for a, b, r, t in zip(A, B, R, T):
        lo, hi = mp.mpf(0), min((mp.mpf(r) / a) ** 0.25, mp.mpf(r) / b)
        for _ in range(200):
            mid = (lo + hi) / 2
            if a * mid ** 4 + b * mid - r > 0:
                hi = mid
            else:
                lo = mid
        assert abs(t - float(lo)) <= 4 * np.spacing(float(lo))
    assert its.max() < 100


def test_quartic_root_special_cases():
    T, _ = quartic_root(0.0, 4.0, 2.0)          # A = 0: linear, T = R/B exactly
    assert T == 0.5
    T, _ = quartic_root(2.0, 0.0, 32.0)         # B = 0: T = (R/A)^(1/4)
    assert abs(T - 2.0) <= 2 * np.spacing(2.0)
    T, _ = quartic_root(1.0, 1.0, -1.0)         # R <= 0: no positive root
    assert T == 0.0
    T, _ = quartic_root(1.0, 1.0, 2.0)          # 1 + 1 = 2 -> T = 1
    assert abs(T - 1.0) <= np.spacing(1.0)


# ---------------------------------------------------------------- prediction (Eq. dis-pre)
def _exact_prediction(P, S):
    """U* of Eq. dis-pre / Eq. dis-pre-marshak with Eq. bc-pre, assembled literally and
    solved by LU in 50-digit arithmetic from the same double inputs (weights
    renormalised to sum exactly to 1 = int_0^1 dv)."""
    mp.mp.dps = 50
    N, M = P.N, P.M
    f = lambda x: mp.mpf(float(x))
    eps, c, a, dt, Cv, dx = f(P.eps), f(P.c), f(P.a), f(P.dt), f(P.Cv), f(P.dx)
    v = [f(x) for x in P.v]
    w = [f(x) for x in P.w]
    sw = sum(w)
    w = [x / sw for x in w]
    T = [f(x) for x in S.T]
    sig = [f(x) for x in P.sig]
    if P.kind == "const":
        kc = [mp.mpf(1)] * N
        kn = [mp.mpf(1)] * (N + 1)
        th = [t ** 3 for t in T]
    else:
        K = [t ** 3 for t in T]
        kc = K
        kn = [0] + [(K[i - 1] + K[i]) / 2 for i in range(1, N)] + [0]
        th = [mp.mpf(1)] * N
    sn = [0] + [2 * sig[i - 1] * sig[i] / (sig[i - 1] + sig[i]) for i in range(1, N)] + [0]
    nE, nO = N * M, (N + 1) * M
    n = nE + nO + N
    A = mp.zeros(n, n)
    b = mp.zeros(n, 1)
    iE = lambda j, k: j * M + k
    iO = lambda i, k: nE + i * M + k
    iU = lambda j: nE + nO + j
    for j in range(N):
        for k in range(M):
            r = iE(j, k)
            A[r, iE(j, k)] += kc[j] / (c * dt) + sig[j] / eps ** 2
            A[r, iO(j + 1, k)] += kc[j] * v[k] / dx
            A[r, iO(j, k)] += -kc[j] * v[k] / dx
            A[r, iU(j)] += -sig[j] * a * c / eps ** 2
            b[r] = kc[j] * f(S.E[j, k]) / (c * dt)
    for i in range(N + 1):
        for k in range(M):
            r = iO(i, k)
            if 1 <= i <= N - 1:
                A[r, iO(i, k)] += kn[i] / (c * dt) + sn[i] / eps ** 2
                A[r, iE(i, k)] += kn[i] * v[k] / (eps ** 2 * dx)
                A[r, iE(i - 1, k)] += -kn[i] * v[k] / (eps ** 2 * dx)
                b[r] = kn[i] * f(S.O[i, k]) / (c * dt)
            elif P.bc == "reflect":
                A[r, iO(i, k)] += 1
            elif i == 0:
                A[r, iO(0, k)] += 1
                A[r, iO(1, k)] += 1
                A[r, iE(0, k)] += 2 / eps
                b[r] = 2 / eps * f(P.bL[k])
            else:
                A[r, iO(N, k)] += 1
                A[r, iO(N - 1, k)] += 1
                A[r, iE(N - 1, k)] += -2 / eps
                b[r] = -2 / eps * f(P.bR[k])
    for j in range(N):
        r = iU(j)
        gg = 4 * sig[j] * th[j] / eps ** 2
        A[r, iU(j)] += Cv / dt + gg * a * c
        for k in range(M):
            A[r, iE(j, k)] += -gg * w[k]
        b[r] = Cv * f(S.U[j]) / dt
    x = mp.lu_solve(A, b)
    U = np.array([float(x[nE + nO + j]) for j in range(N)])
    E = np.array([[float(x[iE(j, k)]) for k in range(M)] for j in range(N)])
    O = np.array([[float(x[iO(i, k)]) for k in range(M)] for i in range(N + 1)])
    return E, O, U


@pytest.mark.parametrize("kind", ["const", "t3"])
@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-5, 1e-8])
@pytest.mark.parametrize("bc", ["inflow", "reflect"])
def test_prediction_matches_50_digit_solution(kind, eps, bc):
    """Eq. dis-pre + Eq. bc-pre (Sec. 4) and Eq. dis-pre-marshak (Sec. 5): the oracle's
    block elimination on (e, rho) equals the literal system solved in 50 digits."""
    P = _problem(N=8, nv=4, eps=eps, kind=kind, bc=bc)
    T = _bumpy_T(P.N)
    S = g.equilibrium_state(P, T)
    rng = np.random.default_rng(2)
    S.E = S.E * (1.0 + 0.05 * rng.standard_normal(S.E.shape))
    S.O = 0.1 * rng.standard_normal(S.O.shape)
    if bc == "reflect":
        S.O[0] = S.O[-1] = 0.0
    E, O, U, rho = g.predict(P, S)
    Ex, Ox, Ux = _exact_prediction(P, S)
    assert np.max(np.abs(U - Ux) / np.abs(Ux)) < 2e-13
    assert np.max(np.abs(E - Ex) / np.abs(Ex)) < 2e-13
    # O near a wall is (2/eps)(b - E) - O: its absolute error grows like u/eps
    tolO = 1e-13 * max(1.0, 1e-2 / eps) * max(1.0, np.max(np.abs(Ox)))
    assert np.max(np.abs(O - Ox)) < tolO


@pytest.mark.parametrize("kind", ["const", "t3"])
@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_prediction_matches_literal_sparse_lu(kind, eps):
    """At eps = O(1) the literal (E, O, U) assembly is well conditioned; both solves agree."""
    P = _problem(N=40, nv=8, eps=eps, kind=kind)
    S = g.equilibrium_state(P, _bumpy_T(P.N, 1))
    S.O = 0.1 * np.random.default_rng(3).standard_normal(S.O.shape)
    E, O, U, _ = g.predict(P, S)
    El, Ol, Ul = g.predict_literal(P, S)
    assert np.max(np.abs(U - Ul) / Ul) < 1e-12
    assert np.max(np.abs(E - El)) / np.max(np.abs(El)) < 1e-12
    assert np.max(np.abs(O - Ol)) / np.max(np.abs(Ol)) < 1e-12


def test_prediction_plants_fail():
    """A dropped term in the literal assembly is caught by the 50-digit pin: perturbing
    the prediction data changes U* well beyond the pin's tolerance."""
    P = _problem(N=8, nv=4, eps=1e-2, kind="t3")
    S = g.equilibrium_state(P, _bumpy_T(P.N))
    _, _, U, _ = g.predict(P, S)
    P2 = _problem(N=8, nv=4, eps=1e-2, kind="t3", bL=1.0 + 1e-9)
    _, _, U2, _ = g.predict(P2, S)
    assert np.max(np.abs(U2 - U) / U) > 1e-11


# ---------------------------------------------------------------- substep 2 (Eq. dis-cor)
@pytest.mark.parametrize("kind", ["const", "t3"])
@pytest.mark.parametrize("eps", [1.0, 1e-3, 1e-6])
def test_substep2_matches_50_digit_solution(kind, eps):
    """Eq. dis-cor1/2 with Eq. dis-cor4 (and Eq. dis-cor-marshak1/2 with Eq. 9171):
    the literal per-angle system, solved in 50 digits."""
    P = _problem(N=8, nv=4, eps=eps, kind=kind)
    rng = np.random.default_rng(4)
    T = _bumpy_T(P.N, 2)
    S = g.equilibrium_state(P, T)
    S.E = S.E * (1 + 0.05 * rng.standard_normal(S.E.shape))
    S.O = rng.standard_normal(S.O.shape)
    Tn = T * (1 + 0.01 * rng.standard_normal(P.N))
    EJ, OJ = g.correct_intensity(P, S, Tn)
    mp.mp.dps = 50
    N, M = P.N, P.M
    f = lambda x: mp.mpf(float(x))
    epsm, c, a, dt, dx = f(P.eps), f(P.c), f(P.a), f(P.dt), f(P.dx)
    U = [f(t) ** 4 for t in Tn]
    if kind == "const":
        kc = [mp.mpf(1)] * N
        kn = [mp.mpf(1)] * (N + 1)
    else:
        K = [f(t) ** 3 for t in Tn]
        kc = K
        kn = [0] + [(K[i - 1] + K[i]) / 2 for i in range(1, N)] + [0]
    sig = [f(s) for s in P.sig]
    sn = [0] + [2 * sig[i - 1] * sig[i] / (sig[i - 1] + sig[i]) for i in range(1, N)] + [0]
    for k in range(M):
        vk = f(P.v[k])
        n = 2 * N + 1
        A = mp.zeros(n, n)
        b = mp.zeros(n, 1)
        for j in range(N):   # cell rows, unknown E_J,j at j ; O_i at N + i
            A[j, j] += kc[j] * epsm / (c * dt) + sig[j] / epsm
            A[j, N + j + 1] += kc[j] * vk / dx
            A[j, N + j] += -kc[j] * vk / dx
            b[j] = kc[j] * (f(S.E[j, k]) - a * c * U[j]) / (c * dt)
        for i in range(N + 1):
            r = N + i
            if 1 <= i <= N - 1:
                A[r, r] += kn[i] / (c * dt) + sn[i] / epsm ** 2
                A[r, i] += kn[i] * vk / (epsm * dx)
                A[r, i - 1] += -kn[i] * vk / (epsm * dx)
                b[r] = kn[i] * f(S.O[i, k]) / (c * dt) - kn[i] * a * c * vk * (U[i] - U[i - 1]) / (epsm ** 2 * dx)
            elif i == 0:
                A[r, N] += 1
                A[r, N + 1] += 1
                A[r, 0] += 2
                b[r] = 2 / epsm * (f(P.bL[k]) - a * c * U[0])
            else:
                A[r, N + N] += 1
                A[r, N + N - 1] += 1
                A[r, N - 1] += -2
                b[r] = 2 / epsm * (a * c * U[N - 1] - f(P.bR[k]))
        x = mp.lu_solve(A, b)
        ej = np.array([float(x[j]) for j in range(N)])
        En_new = P.a * P.c * Tn ** 4 + P.eps * EJ[:, k]
        Ex_new = np.array([float(a * c * U[j] + epsm * x[j]) for j in range(N)])
        assert np.max(np.abs(En_new - Ex_new) / np.abs(Ex_new)) < 1e-13
        ox = np.array([float(x[N + i]) for i in range(N + 1)])
        assert np.max(np.abs(OJ[:, k] - ox)) <= 1e-12 * max(1.0, np.max(np.abs(ox)))


# ---------------------------------------------------------------- invariants of Algorithm 2
@pytest.mark.parametrize("kind", ["const", "t3"])
@pytest.mark.parametrize("eps", [1.0, 1e-3, 1e-6])
def test_equilibrium_preserved(kind, eps):
    """Uniform T, I = acT^4 and inflow b = acT^4: E* = acU^n, O* = 0 solve Eq. dis-pre,
    R = A T^4 + B T^n in Eq. Tnp1 gives T^{n+1} = T^n, and Eq. dis-cor has zero data,
    so the state is a fixed point of Algorithm 2."""
    T0 = 0.7
    P = _problem(N=16, nv=8, eps=eps, kind=kind, sig=3.0, bL=T0 ** 4, bR=T0 ** 4)
    S = g.equilibrium_state(P, np.full(P.N, T0))
    for _ in range(3):
        S = g.step(P, S)
    # the wall cells see (2/eps)(b - E) through Eq. bc-pre: rounding grows like u/eps there
    tol = 1e-14 + 5e-16 / eps
    assert np.max(np.abs(S.T - T0)) < tol
    assert np.max(np.abs(S.E - T0 ** 4)) < tol
    # I(+-v) = E +- eps O: the odd part's contribution to I stays at rounding level
    assert np.max(np.abs(P.eps * S.O)) < tol


@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-4])
def test_total_energy_conserved_reflecting(eps):
    """Eq. semiconservative summed over cells: with reflecting walls and a uniform,
    T-independent sigma the flux terms telescope to zero, so
    sum_j dx (rho_j/c + Cv T_j) is constant."""
    P = _problem(N=32, nv=8, eps=eps, kind="const", sig=2.0, bc="reflect")
    S = g.equilibrium_state(P, _bumpy_T(P.N, 7) + 0.2)
    e0 = g.energy(P, S)
    for _ in range(5):
        S = g.step(P, S)
        assert abs(g.energy(P, S) - e0) < 1e-13 * e0


@pytest.mark.parametrize("eps", [1.0, 1e-2, 1e-4])
def test_per_cell_energy_identity(eps):
    """Eq. semiconservative in 1D, cell by cell (any T-independent sigma(x), inflow walls):
    (rho^{n+1}-rho^n)/(c dt) + Cv (T^{n+1}-T^n)/dt + F*/dx
        - eps^2/(c sigma dt + eps^2) (F* - F^{n+1})/dx = 0,
    F = sum_k w_k v_k (O_{j+1,k} - O_{j,k})."""
    x = (np.arange(40) + 0.5) / 40
    sig = np.where(((x >= 0.2) & (x <= 0.35)) | ((x >= 0.65) & (x <= 0.8)), 0.2, 1.0)  # Eq. eqn:sigma
    P = _problem(N=40, nv=8, eps=eps, kind="const", sig=sig)
    S = g.equilibrium_state(P, _bumpy_T(P.N, 8) + 0.1)
    info = g.StepInfo()
    S1 = g.step(P, S, info)
    c, dt, dx, Cv = P.c, P.dt, P.dx, P.Cv
    rho0, rho1 = g.rho_of(P, S.E), g.rho_of(P, S1.E)
    F1 = g.flux_div(P, S1.O)
    Fs = info.Fstar
    terms = [(rho1 - rho0) / (c * dt), Cv * (S1.T - S.T) / dt, Fs / dx,
             -eps ** 2 / (c * sig * dt + eps ** 2) * (Fs - F1) / dx]
    res = sum(terms)
    scale = sum(np.abs(t) for t in terms) + np.abs(rho0) / (c * dt)
    assert np.max(np.abs(res) / scale) < 1e-13


def test_energy_identity_catches_planted_sign_error():
    """The per-cell identity fails if the right-wall sign of the projection's boundary
    row is flipped (the reading the paper's Eq. dis-proj display would give)."""
    P = _problem(N=20, nv=4, eps=1e-2, kind="const", bL=0.3, bR=0.9)
    S = g.equilibrium_state(P, _bumpy_T(P.N, 9) + 0.1)
    info = g.StepInfo()
    S1 = g.step(P, S, info)
    bad = S1.O.copy()
    bad[-1] = 2.0 / P.eps * (P.bR - S1.E[-1]) - S1.O[-2]
    F_good = g.flux_div(P, S1.O)
    F_bad = g.flux_div(P, bad)
    assert np.max(np.abs(F_bad - F_good)) > 1.0


# ---------------------------------------------------------------- limits
def test_diffusion_limit_prediction_and_correction():
    """Sec. 4 diffusion limits (Eq. 9162 and the limit of Eq. dis-cor): at eps -> 0 with
    I = acT^4 the prediction's U* is the three-stage solver's stage 1 (Eq. dis-diff)
    up to O(eps^2) and T^{n+1} is its stage 2 up to O(eps).  Reflecting walls on both
    (zero flux in the limit)."""
    N = 32
    x = (np.arange(N) + 0.5) / N
    T = np.maximum(1 - 40 * (x - 0.5) ** 2, 0.0) + 0.05   # Eq. IC000, lifted off zero
    P = _problem(N=N, nv=16, eps=1e-7, kind="const", sig=1.0, bc="reflect", cfl=0.1)
    S = g.equilibrium_state(P, T)
    info = g.StepInfo()
    g.step(P, S, info)
    Td, Ud = dif.three_stage_step(T, P.sig, P.dx, P.dt, kind="const")
    assert np.max(np.abs(info.Ustar - Ud) / Ud) < 1e-9
    assert np.max(np.abs(info.T_new - Td) / Td) < 1e-5
    # and the two-stage variant differs at O(dt) (the paper's front argument, Eq. dis-diff-2)
    T2 = dif.two_stage_step(T, P.sig, P.dx, P.dt)
    assert np.max(np.abs(T2 - Td) / Td) > 1e-4


def test_diffusion_limit_prediction_sigma_T3():
    """Sec. 5: the sigma/T^3 prediction tends to the first line of Eq. marshak-diff2."""
    N = 32
    x = (np.arange(N) + 0.5) / N
    T = np.maximum(1 - 40 * (x - 0.5) ** 2, 0.0) + 0.05
    P = _problem(N=N, nv=16, eps=1e-7, kind="t3", sig=1.0, bc="reflect", cfl=0.1)
    S = g.equilibrium_state(P, T)
    _, _, U, _ = g.predict(P, S)
    _, Ud = dif.three_stage_step(T, P.sig, P.dx, P.dt, kind="t3")
    assert np.max(np.abs(U - Ud) / Ud) < 1e-9


def test_front_moves_with_three_stages_not_two():
    """Remark after Eq. dis-diff: from compactly supported data the two-stage scheme
    keeps T = 0 where it was 0; the three-stage scheme moves the front."""
    N = 50
    x = (np.arange(N) + 0.5) / N
    T = np.maximum(1 - 40 * (x - 0.5) ** 2, 0.0)       # Eq. IC000
    dx, dt = 1.0 / N, 0.05 / N
    T3, T2 = T.copy(), T.copy()
    for _ in range(40):
        T3, _ = dif.three_stage_step(T3, np.ones(N), dx, dt)
        T2 = dif.two_stage_step(T2, np.ones(N), dx, dt)
    zero = T == 0
    assert np.all(T2[zero] == 0.0)
    assert np.any(T3[zero] > 1e-3)


def test_three_stage_tracks_implicit_solver():
    """Sec. 6.1 (Eq. imp_T as reference): same grid, dt = 0.05 dx, striped sigma of
    Eq. eqn:sigma with sigma_0 = 0.2 - agreement to the first-order error."""
    N = 100
    x = (np.arange(N) + 0.5) / N
    T = np.maximum(np.sin(2 * np.pi * (x - 0.25)), 0.0) ** 0.25
    sig = np.where(((x >= 0.2) & (x <= 0.35)) | ((x >= 0.65) & (x <= 0.8)), 0.2, 1.0)
    dx = 1.0 / N
    dt = 0.05 * dx
    T3, Ti = T.copy(), T.copy()
    for _ in range(200):
        T3, _ = dif.three_stage_step(T3, sig, dx, dt)
        Ti = dif.implicit_T4_step(Ti, sig, dx, dt)
    assert np.max(np.abs(T3 - Ti)) < 2e-2
    assert np.sum(np.abs(T3 - Ti)) * dx < 2e-3


def test_free_streaming_first_order():
    """sigma = 0, eps = 1 (the free-streaming limit of the abstract): the scheme
    approaches the exact characteristic solution I(t,x,v) = I_in(x - c v t, v) with
    error decreasing at least at first order in dx (Sec. 6.2 reports first order)."""
    from paper_1811_05579_gb300 import workloads as wl
    _, alpha, phi = wl.free_streaming_1d()
    errs = []
    for N in (32, 64, 128):
        v, w = gauss_legendre_half(8)
        P = g.Problem(N=N, v=v, w=w, sig=0.0, eps=1.0, dt=0.25 / N, kind="const",
                      bL=wl.free_streaming_intensity(0.0, v, alpha, phi),
                      bR=wl.free_streaming_intensity(1.0, -v, alpha, phi))
        xc = (np.arange(N) + 0.5) / N
        Ip = wl.free_streaming_intensity(xc[:, None], v[None, :], alpha, phi)
        In = wl.free_streaming_intensity(xc[:, None], -v[None, :], alpha, phi)
        S = g.state_from_intensity(P, np.ones(N), Ip, In)
        nsteps = N // 4          # t = 1/16
        S = g.run(P, S, nsteps)
        t = nsteps * P.dt
        # exact: follow the characteristic back; inflow value once it leaves the slab
        xs = xc[:, None] - v[None, :] * t
        Ipx = np.where(xs >= 0, wl.free_streaming_intensity(xs, v[None, :], alpha, phi),
                       wl.free_streaming_intensity(0.0, v[None, :], alpha, phi))
        xs2 = xc[:, None] + v[None, :] * t
        Inx = np.where(xs2 <= 1, wl.free_streaming_intensity(xs2, -v[None, :], alpha, phi),
                       wl.free_streaming_intensity(1.0, -v[None, :], alpha, phi))
        Ipn, Inn = g.intensity(P, S)
        errs.append(np.mean(np.abs(Ipn - Ipx)) + np.mean(np.abs(Inn - Inx)))
        assert np.max(np.abs(S.T - 1.0)) == 0.0      # sigma = 0: T frozen exactly
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 0.8, (errs, rates)


# ---------------------------------------------------------------- learned-guess network (oracle)
def test_mlp_oracle_backprop_matches_finite_differences():
    """The FP64 backpropagation of oracle/mlp.py against central differences of its own
    loss (weights kept in FP64 here, so the derivative is exact up to O(h^2))."""
    from oracle import mlp as om
    rng = np.random.default_rng(11)
    p = 0.3 * rng.standard_normal(om.N_PARAMS)
    x = rng.standard_normal((7, om.N_IN))
    t = rng.standard_normal(7)
    loss, g = om.loss_and_grad(p, x, t, bf16=False)
    idx = rng.choice(om.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [om.N_PARAMS - 1, 0]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (om.loss_and_grad(p + e, x, t, bf16=False)[0] - om.loss_and_grad(p - e, x, t, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding_is_nearest_even():
    from oracle import mlp as om
    assert om.to_bf16(np.float32(1.0)) == 1.0
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7 in bf16: ties to even (1.0)
    assert om.to_bf16(np.float32(1.0 + 2 ** -8)) == 1.0
    assert om.to_bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6
    assert om.to_bf16(np.float32(-2.5)) == -2.5
