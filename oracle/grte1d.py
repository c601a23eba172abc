"""1D fully discrete AP scheme for the gray radiative transfer equation (oracle).

TEST INFRASTRUCTURE ONLY - see oracle/__init__.py.

Follows Algorithm 2 (Sec. 4) for a temperature-independent opacity sigma(x) and its
sigma/T^3 form (Sec. 5), the latter for a general exponent sigma_0/T^p (Problem.p, 3 by
default; the paper treats p = 3 and names other nonlinearities as extensions, Sec. 1 and
Sec. 5).  Notation (0-based):

  cells  j = 0..N-1 at x_{j+1/2}: E[j, k], U[j], T[j]          (Eq. E000)
  nodes  i = 0..N   at x_i = i dx: O[i, k]                      (Eq. O000)
  angles k = 0..M-1, v_k > 0, weights w_k with sum w_k = int_0^1 dv = 1.

Node i sits between cell i-1 and cell i.  E = (I(v) + I(-v))/2 and
O = (I(v) - I(-v))/(2 eps) (Eq. EO), so I(+v) = E + eps O and I(-v) = E - eps O.

Both opacity forms are written with two per-cell multipliers:

  kappa  multiplies the time-derivative and streaming terms: 1 for sigma(x);
         K = T^p for sigma/T^p (Eq. dis-pre-marshak, "multiplied to the left hand
         side"), with node values K_i = (K_{i-1/2} + K_{i+1/2})/2.
  theta  multiplies sigma in the U equation: T^3 for sigma(x) (Eq. dis-pre3), T^{3-p}
         for sigma/T^p (1 at p = 3: third line of Eq. dis-pre-marshak; the factor
         4 T^3 of dU = 4 T^3 dT over the T^p the equation was multiplied by).
  In the correction, V* = max(U*, 0)^{p/4} (= (T^{n+1*})^p) takes the place of
  (U*)^{3/4}.  p = 0 gives back the sigma(x) scheme exactly; 0 <= p <= 3.

and "sig" is sigma(x) (or sigma_0(x) of sigma_0/T^3), given per cell.  Node values
of sig are the harmonic mean of the two neighbouring cells (the paper evaluates
sigma_i without saying how; the harmonic mean matches the (1/sigma) averaging of
Eq. diff_solver).

Boundary conditions: 'inflow' is Eq. bc-pre (left: I(0, v) = b_L(v); right:
I(L, -v) = b_R(-v)); 'reflect' sets the odd part to zero at the wall node
(I(v) = I(-v) there).

Linear solves: the prediction is solved by block-tridiagonal Gaussian elimination
on the unknowns (e, rho) of coefficients() - an exact rewrite of the paper's
equations with E = rho + e that avoids the O(1/eps^2) cancellation of the literal
(E, O, U) form; predict_literal() keeps the literal assembly (sparse LU) as a check.
The correction substep 2 is assembled literally and solved by sparse LU.  The
quadrature weights enter as exactly normalised (sum_k w_k = 1 = int_0^1 dv): the
prediction's isotropic balance is sensitive at O(u/eps^2) to a rounding error in
that sum.
"""
from dataclasses import dataclass, field
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .scalar import quartic_root

SIGMA_CONST = "const"   # sigma(x), independent of T
SIGMA_T3 = "t3"         # sigma_0(x) / T^p (p = 3 unless Problem.p says otherwise)


@dataclass
class Problem:
    """Static data of one 1D instance (cells on [x0, x1], uniform)."""
    N: int
    v: np.ndarray            # (M,) positive angles
    w: np.ndarray            # (M,) weights, sum = 1
    sig: np.ndarray          # (N,) sigma(x) or sigma_0(x) per cell
    a: float = 1.0
    c: float = 1.0
    Cv: float = 1.0
    eps: float = 1.0
    dt: float = 1e-3
    kind: str = SIGMA_CONST
    bc: str = "inflow"       # 'inflow' or 'reflect'
    bL: np.ndarray = None    # (M,) inflow I(0, +v_k)
    bR: np.ndarray = None    # (M,) inflow I(L, -v_k)
    x0: float = 0.0
    x1: float = 1.0
    p: float = 3.0           # the exponent of sigma_0/T^p (kind 't3')

    def __post_init__(self):
        self.v = np.asarray(self.v, dtype=np.float64)
        self.w = np.asarray(self.w, dtype=np.float64)
        self.sig = np.broadcast_to(np.asarray(self.sig, dtype=np.float64), (self.N,)).copy()
        M = self.v.size
        if self.bL is None:
            self.bL = np.zeros(M)
        if self.bR is None:
            self.bR = np.zeros(M)
        self.bL = np.broadcast_to(np.asarray(self.bL, dtype=np.float64), (M,)).copy()
        self.bR = np.broadcast_to(np.asarray(self.bR, dtype=np.float64), (M,)).copy()

    @property
    def M(self):
        return self.v.size

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.N

    def node_sig(self):
        """sig at interior nodes i = 1..N-1 (harmonic mean of the two cells)."""
        s = self.sig
        out = np.zeros(self.N + 1)
        l, r = s[:-1], s[1:]
        with np.errstate(divide="ignore", invalid="ignore"):
            h = np.where((l > 0) & (r > 0), 2.0 * l * r / (l + r), 0.0)
        out[1:-1] = h
        return out


@dataclass
class State:
    E: np.ndarray   # (N, M)
    O: np.ndarray   # (N+1, M)
    U: np.ndarray   # (N,)
    T: np.ndarray   # (N,)
    t: float = 0.0
    step: int = 0


@dataclass
class StepInfo:
    """Intermediate results of one step, kept for tests."""
    Estar: np.ndarray = None
    Ostar: np.ndarray = None
    Ustar: np.ndarray = None
    Fstar: np.ndarray = None     # sum_k w_k v_k (O*_{j+1,k} - O*_{j,k}) per cell
    rho_n: np.ndarray = None
    T_new: np.ndarray = None
    newton_its: np.ndarray = None
    EJ: np.ndarray = None
    negative_R: int = 0
    extra: dict = field(default_factory=dict)


def equilibrium_state(P, T):
    """I = a c T^4 (Q10 reading of the initial data): E = acT^4, O = 0, U = T^4."""
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (P.N,)).copy()
    U = T ** 4
    E = np.repeat((P.a * P.c * U)[:, None], P.M, axis=1)
    O = np.zeros((P.N + 1, P.M))
    return State(E=E, O=O, U=U, T=T)


def state_from_intensity(P, T, Ipos, Ineg):
    """Even/odd parts (Eq. EO) of given cell-centre intensities I(+v_k), I(-v_k).

    O lives on nodes: interior node values are the mean of the two neighbouring
    cells' odd parts; wall nodes copy the adjacent cell.
    """
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (P.N,)).copy()
    E = 0.5 * (Ipos + Ineg)
    Oc = (Ipos - Ineg) / (2.0 * P.eps)
    O = np.zeros((P.N + 1, P.M))
    O[1:-1] = 0.5 * (Oc[:-1] + Oc[1:])
    O[0] = Oc[0]
    O[-1] = Oc[-1]
    return State(E=E, O=O, U=T ** 4, T=T)


def _multipliers(P, T):
    """(kappa_cell, kappa_node, theta) for the given temperature (see module doc)."""
    N = P.N
    if P.kind == SIGMA_CONST:
        kc = np.ones(N)
        kn = np.ones(N + 1)
        theta = T ** 3
    elif P.kind == SIGMA_T3:
        K = T ** P.p
        kc = K
        kn = np.zeros(N + 1)
        kn[1:-1] = 0.5 * (K[:-1] + K[1:])
        theta = T ** (3.0 - P.p)
    else:
        raise ValueError(P.kind)
    return kc, kn, theta


def rho_of(P, E):
    """rho = <I> = int_0^1 E dv = sum_k w_k E_k per cell."""
    return E @ P.w


def flux_div(P, O):
    """sum_k w_k v_k (O_{j+1,k} - O_{j,k}) per cell (the angular integral in Eq. Tnp1)."""
    return (O[1:] - O[:-1]) @ (P.w * P.v)


def coefficients(P, T):
    """Per-cell / per-node coefficients of the prediction system at temperature T.

    With E = rho + e (rho = sum_k w_k E_k, so sum_k w_k e_k = 0) the prediction
    system of Eq. dis-pre / Eq. dis-pre-marshak is rewritten, without approximation,
    as

      e-equation (cell j, angle k):
        A_j e_k + (G_k (rho + e_k))_j + phi_jk = kappa_j (E^n_jk - rho_j)/(c dt) - s_j (rho_j - a c U^n_j)
      conservation (cell j):
        alpha_j rho_j + sum_k w_k [(G_k (rho + e_k))_j + phi_jk] = kappa_j rho^n_j/(c dt) + s_j a c U^n_j

    where U* has been eliminated with Eq. dis-pre3 (as the paper prescribes):
      sig (a c U* - rho)/eps^2 = -s (rho - a c U^n),  s = sig Cv/(Cv eps^2 + 4 sig theta dt a c),
      U* = (U^n + gam rho)/(1 + gam a c),  gam = 4 sig theta dt/(eps^2 Cv),
    O has been eliminated with the node equation (Eq. dis-pre1) and Eq. bc-pre:
      O_i = o_i - d_i v (E_i - E_{i-1})/dx  (interior node i),
      o_i = d_i eps^2 O^n_i/(c dt),  d_i = kappa_i/(kappa_i eps^2/(c dt) + sig_i),
    and kappa v (O_{j+1} - O_j)/dx = (G_k E)_j + phi_jk splits the streaming term into
    its part linear in E (G_k = v^2 Gint + v Gbdry, tridiagonal) and its data part.
    A = kappa/(c dt) + sig/eps^2 and alpha = kappa/(c dt) + s.  The conservation
    equation is the v-average of the cell equations plus Eq. dis-pre3; it replaces the
    closure sum_k w_k e_k = 0, which it implies.  Solving for rho and e (rather than
    for E and U directly) keeps the isotropic balance free of the O(1/eps^2)
    cancellation between sig E/eps^2 and sig a c U/eps^2.
    """
    N = P.N
    eps, c, a, dt, dx, Cv = P.eps, P.c, P.a, P.dt, P.dx, P.Cv
    kc, kn, theta = _multipliers(P, T)
    sc = P.sig
    sn = P.node_sig()
    s = sc * Cv / (Cv * eps ** 2 + 4.0 * sc * theta * dt * a * c)
    gam = 4.0 * sc * theta * dt / (eps ** 2 * Cv)
    d = np.zeros(N + 1)
    d[1:-1] = kn[1:-1] / (kn[1:-1] * eps ** 2 / (c * dt) + sn[1:-1])
    inflow = P.bc == "inflow"
    mR = np.ones(N)
    mL = np.ones(N)
    if inflow:
        mR[0] = 2.0        # O_1 - O_0 = 2 O_1 + 2/eps (E_0 - b_L)
        mL[N - 1] = 2.0    # O_N - O_{N-1} = 2/eps (E_{N-1} - b_R) - 2 O_{N-1}
    gl = np.zeros(N)
    gu = np.zeros(N)
    gb = np.zeros(N)
    gu[:N - 1] = kc[:N - 1] * mR[:N - 1] * d[1:N] / dx ** 2
    gl[1:] = kc[1:] * mL[1:] * d[1:N] / dx ** 2
    if inflow:
        gb[0] += 2.0 * kc[0] / (eps * dx)
        gb[N - 1] += 2.0 * kc[N - 1] / (eps * dx)
    return dict(kc=kc, kn=kn, theta=theta, s=s, gam=gam, d=d, gl=gl, gu=gu, gb=gb,
                gd=gl + gu, A=kc / (c * dt) + sc / eps ** 2, alpha=kc / (c * dt) + s,
                mR=mR, mL=mL)


def _phi(P, C, Oold, bL, bR):
    """Data part phi_jk of kappa v (O_{j+1} - O_j)/dx (see coefficients())."""
    N = P.N
    eps, c, dt, dx = P.eps, P.c, P.dt, P.dx
    o = np.zeros((N + 1, P.M))
    o[1:-1] = (C["d"][1:-1] * eps ** 2 / (c * dt))[:, None] * Oold[1:-1]
    diff = o[1:] - o[:-1]
    if P.bc == "inflow":
        diff[0] = 2.0 * o[1] - 2.0 / eps * bL
        diff[N - 1] = -2.0 / eps * bR - 2.0 * o[N - 1]
    return (C["kc"] / dx)[:, None] * P.v[None, :] * diff, o


def predict(P, S):
    """Prediction (Eq. dis-pre / Eq. dis-pre-marshak with Eq. bc-pre) solved exactly by
    block-tridiagonal Gaussian elimination (dense (M+1)x(M+1) blocks, partial
    pivoting inside each block) on the unknowns z_j = (e_j0..e_j,M-1, rho_j) of
    coefficients().  Returns (E*, O*, U*, rho*)."""
    N, M = P.N, P.M
    eps, c, a, dt, dx = P.eps, P.c, P.a, P.dt, P.dx
    v, w = P.v, P.w
    C = coefficients(P, S.T)
    phi, o = _phi(P, C, S.O, P.bL, P.bR)
    rho_n = S.E @ w
    v2 = v ** 2
    wv2 = np.sum(w * v2)
    idx = np.arange(M)
    Ls = np.zeros((N, M + 1, M + 1))
    Us = np.zeros((N, M + 1, M + 1))
    Ds = np.zeros((N, M + 1, M + 1))
    Rs = np.zeros((N, M + 1))
    for j in range(N):
        gk = v2 * C["gd"][j] + v * C["gb"][j]
        D = Ds[j]
        D[idx, idx] = C["A"][j] + gk
        D[:M, M] = C["alpha"][j] + gk
        D[M, :M] = w * gk
        D[M, M] = C["alpha"][j] + np.sum(w * gk)
        for Mat, coef in ((Ls[j], C["gl"][j]), (Us[j], C["gu"][j])):
            Mat[idx, idx] = -v2 * coef
            Mat[:M, M] = -v2 * coef
            Mat[M, :M] = -w * v2 * coef
            Mat[M, M] = -wv2 * coef
        Rs[j, :M] = C["kc"][j] * S.E[j] / (c * dt) + C["s"][j] * a * c * S.U[j] - phi[j]
        Rs[j, M] = C["kc"][j] * rho_n[j] / (c * dt) + C["s"][j] * a * c * S.U[j] - np.sum(w * phi[j])
    # forward elimination and back substitution (block Thomas)
    SU = np.zeros((N, M + 1, M + 1))
    y = np.zeros((N, M + 1))
    for j in range(N):
        Sj = Ds[j].copy()
        rj = Rs[j].copy()
        if j > 0:
            Sj -= Ls[j] @ SU[j - 1]
            rj -= Ls[j] @ y[j - 1]
        SU[j] = np.linalg.solve(Sj, Us[j])
        y[j] = np.linalg.solve(Sj, rj)
    z = np.zeros((N, M + 1))
    z[N - 1] = y[N - 1]
    for j in range(N - 2, -1, -1):
        z[j] = y[j] - SU[j] @ z[j + 1]
    rho = z[:, M]
    e = z[:, :M]
    E = rho[:, None] + e
    # O* from Eq. dis-pre1 (interior nodes, with E_i - E_{i-1} taken on the split
    # rho + e) and Eq. bc-pre (walls)
    O = np.zeros((N + 1, M))
    dE = (rho[1:] - rho[:-1])[:, None] + (e[1:] - e[:-1])
    O[1:-1] = o[1:-1] - C["d"][1:-1, None] * v[None, :] * dE / dx
    if P.bc == "inflow":
        O[0] = 2.0 / eps * ((P.bL - rho[0]) - e[0]) - O[1]
        O[N] = 2.0 / eps * ((rho[N - 1] - P.bR) + e[N - 1]) - O[N - 1]
    U = (S.U + C["gam"] * rho) / (1.0 + C["gam"] * a * c)
    return E, O, U, rho


def predict_literal(P, S):
    """Prediction assembled literally from Eq. dis-pre (or Eq. dis-pre-marshak) and
    Eq. bc-pre in the unknowns (E*, O*, U*) and solved by sparse LU.  Accurate only
    while eps is not small (the isotropic balance is an O(1/eps^2) cancellation in
    these unknowns); kept as an independent check of predict()."""
    N, M = P.N, P.M
    eps, c, a, dt, dx, Cv = P.eps, P.c, P.a, P.dt, P.dx, P.Cv
    v, w = P.v, P.w
    kc, kn, theta = _multipliers(P, S.T)
    sc = P.sig
    sn = P.node_sig()

    nE = N * M
    nO = (N + 1) * M
    n = nE + nO + N
    iE = lambda j, k: j * M + k
    iO = lambda i, k: nE + i * M + k
    iU = lambda j: nE + nO + j

    rows, cols, vals = [], [], []
    b = np.zeros(n)

    def add(r, cidx, val):
        rows.append(r)
        cols.append(cidx)
        vals.append(val)

    for j in range(N):
        for k in range(M):
            # Cell equation (Eq. dis-pre2 / second line of Eq. dis-pre-marshak):
            # kappa/(c dt) (E - E^n) + kappa v (O_{j+1} - O_j)/dx = sig/eps^2 (a c U - E)
            r = iE(j, k)
            add(r, iE(j, k), kc[j] / (c * dt) + sc[j] / eps ** 2)
            add(r, iO(j + 1, k), kc[j] * v[k] / dx)
            add(r, iO(j, k), -kc[j] * v[k] / dx)
            add(r, iU(j), -sc[j] * a * c / eps ** 2)
            b[r] = kc[j] * S.E[j, k] / (c * dt)
    for i in range(N + 1):
        for k in range(M):
            r = iO(i, k)
            if 1 <= i <= N - 1:
                # Node equation (Eq. dis-pre1 / first line of Eq. dis-pre-marshak):
                # kappa/(c dt)(O - O^n) + kappa v (E_i - E_{i-1})/(eps^2 dx) = -sig O/eps^2
                add(r, iO(i, k), kn[i] / (c * dt) + sn[i] / eps ** 2)
                add(r, iE(i, k), kn[i] * v[k] / (eps ** 2 * dx))
                add(r, iE(i - 1, k), -kn[i] * v[k] / (eps ** 2 * dx))
                b[r] = kn[i] * S.O[i, k] / (c * dt)
            elif P.bc == "reflect":
                add(r, iO(i, k), 1.0)
            elif i == 0:
                # Eq. bc-pre, left: O_0 = 2/eps (b_L - E_0) - O_1
                add(r, iO(0, k), 1.0)
                add(r, iO(1, k), 1.0)
                add(r, iE(0, k), 2.0 / eps)
                b[r] = 2.0 / eps * P.bL[k]
            else:
                # Eq. bc-pre, right: O_N = 2/eps (E_{N-1} - b_R) - O_{N-1}
                add(r, iO(N, k), 1.0)
                add(r, iO(N - 1, k), 1.0)
                add(r, iE(N - 1, k), -2.0 / eps)
                b[r] = -2.0 / eps * P.bR[k]
    for j in range(N):
        # U equation (Eq. dis-pre3 / third line of Eq. dis-pre-marshak):
        # Cv (U - U^n)/dt = 4 sig theta/eps^2 (sum_k w_k E_k - a c U)
        r = iU(j)
        g = 4.0 * sc[j] * theta[j] / eps ** 2
        add(r, iU(j), Cv / dt + g * a * c)
        for k in range(M):
            add(r, iE(j, k), -g * w[k])
        b[r] = Cv * S.U[j] / dt

    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    x = spla.spsolve(A, b)
    E = x[:nE].reshape(N, M)
    O = x[nE:nE + nO].reshape(N + 1, M)
    U = x[nE + nO:]
    return E, O, U


def correction_temperature(P, S, Fstar, Ustar):
    """Correction substep 1: per-cell scalar equation for T^{n+1}; Fstar is the flux of
    correction_flux().

    sigma(x): Eq. Tnp1,
      1/(c dt) [a c T^4 + eps^2 Cv/(sig dt) (T - T^n)] + Cv/dt (T - T^n)
          = rho^n/(c dt) - Fstar/dx.
    sigma/T^3: the sum of Eq. dis-cor-marshak4 and Eq. dis-cor-marshak5 over v, i.e.
      the same with eps^2 Cv/(sig dt) replaced by eps^2 K* Cv/(sig_0 dt),
      K* = (U*)^{3/4} (U* < 0 read as 0).
    Both are multiplied through by sig so that sig = 0 stays finite:
      A T^4 + B T = R,  A = sig a/dt,  B = sig Cv/dt + eps^2 kap Cv/(c dt^2),
      R = sig (rho^n/(c dt) - Fstar/dx) + B T^n,  kap = 1 or K*.
    """
    eps, c, a, dt, dx, Cv = P.eps, P.c, P.a, P.dt, P.dx, P.Cv
    sig = P.sig
    rho_n = rho_of(P, S.E)
    if P.kind == SIGMA_CONST:
        kap = np.ones(P.N)
    else:
        kap = np.maximum(Ustar, 0.0) ** (P.p / 4.0)
    A = sig * a / dt
    B = sig * Cv / dt + eps ** 2 * kap * Cv / (c * dt ** 2)
    R = sig * (rho_n / (c * dt) - Fstar / dx) + B * S.T
    T, its = quartic_root(A, B, R)
    undetermined = np.isnan(T)
    T = np.where(undetermined, S.T, T)
    return T, its, int(np.sum(R <= 0.0) - np.sum(undetermined & (R <= 0.0))), rho_n


def correct_intensity(P, S, Tnew):
    """Correction substep 2: Eq. dis-cor1/dis-cor2 with Eq. dis-cor4 (sigma(x)) or
    Eq. dis-cor-marshak1/2 with Eq. 9171 (sigma/T^3), U^{n+1*} replaced by
    (T^{n+1})^4, K^{n+1*} by (T^{n+1})^3 and the starred E_J, O_J by the new ones;
    boundary rows as in the boundary conditions of the correction step.
    Returns (E_J, O_J)."""
    N, M = P.N, P.M
    eps, c, a, dt, dx = P.eps, P.c, P.a, P.dt, P.dx
    v = P.v
    U = Tnew ** 4
    if P.kind == SIGMA_CONST:
        kc = np.ones(N)
        kn = np.ones(N + 1)
    else:
        K = Tnew ** P.p
        kc = K
        kn = np.zeros(N + 1)
        kn[1:-1] = 0.5 * (K[:-1] + K[1:])
    sc = P.sig
    sn = P.node_sig()

    nE = N * M
    nO = (N + 1) * M
    n = nE + nO
    iE = lambda j, k: j * M + k
    iO = lambda i, k: nE + i * M + k
    rows, cols, vals = [], [], []
    b = np.zeros(n)

    def add(r, cidx, val):
        rows.append(r)
        cols.append(cidx)
        vals.append(val)

    for j in range(N):
        for k in range(M):
            # kappa/(c dt) (a c U + eps E_J - E^n) + kappa v (O_{j+1} - O_j)/dx = -sig E_J/eps
            r = iE(j, k)
            add(r, iE(j, k), kc[j] * eps / (c * dt) + sc[j] / eps)
            add(r, iO(j + 1, k), kc[j] * v[k] / dx)
            add(r, iO(j, k), -kc[j] * v[k] / dx)
            b[r] = kc[j] * (S.E[j, k] - a * c * U[j]) / (c * dt)
    for i in range(N + 1):
        for k in range(M):
            r = iO(i, k)
            if 1 <= i <= N - 1:
                # kappa/(c dt)(O - O^n) + kappa a c v (U_i - U_{i-1})/(eps^2 dx)
                #   + kappa v (E_J,i - E_J,i-1)/(eps dx) = -sig O/eps^2
                add(r, iO(i, k), kn[i] / (c * dt) + sn[i] / eps ** 2)
                add(r, iE(i, k), kn[i] * v[k] / (eps * dx))
                add(r, iE(i - 1, k), -kn[i] * v[k] / (eps * dx))
                b[r] = kn[i] * S.O[i, k] / (c * dt) - kn[i] * a * c * v[k] * (U[i] - U[i - 1]) / (eps ** 2 * dx)
            elif P.bc == "reflect":
                add(r, iO(i, k), 1.0)
            elif i == 0:
                # O_0 = 2/eps (b_L - E_0) - O_1 with E_0 = a c U_0 + eps E_J,0
                add(r, iO(0, k), 1.0)
                add(r, iO(1, k), 1.0)
                add(r, iE(0, k), 2.0)
                b[r] = 2.0 / eps * (P.bL[k] - a * c * U[0])
            else:
                # O_N = 2/eps (E_{N-1} - b_R) - O_{N-1}
                add(r, iO(N, k), 1.0)
                add(r, iO(N - 1, k), 1.0)
                add(r, iE(N - 1, k), -2.0)
                b[r] = 2.0 / eps * (a * c * U[N - 1] - P.bR[k])
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    x = spla.spsolve(A, b)
    EJ = x[:nE].reshape(N, M)
    OJ = x[nE:].reshape(N + 1, M)
    return EJ, OJ


def correction_flux(P, S, Es, Os, Us):
    """The flux sum_k w_k v_k (O_{J,j+1} - O_{J,j}) that the temperature equation of the
    correction takes from the predicted state.

    sigma(x): O_J^{n+1*} = O^{n+1*}, the prediction's own O (stated after Eq. Tnp1).
    sigma/T^3: Eq. dis-cor-marshak1 evaluated with the predicted data, i.e. the node
    flux with the multiplier V* = (U*)^{3/4} (node values the mean of the two cells,
    U* < 0 read as 0) in place of the prediction's K^n = (T^n)^3:
        O~_i = d*_i [eps^2 O^n_i/(c dt) - v (E*_i - E*_{i-1})/dx],
        d*_i = V*_i/(V*_i eps^2/(c dt) + sig_i)   (interior nodes).
    This is the reading under which the correction's diffusion limit carries
    (T^{n+1*})^3 as the remark closing Sec. 5 states (with K^n frozen at T^n the two
    coincide only for sigma(x)); it is also the one that reproduces the Marshak front of
    Sec. 6.5 at eps = 1e-5.
    Inflow walls (the paper gives Eq. dis-cor-marshak1 for the interior nodes only): the
    wall node takes the prediction's wall value shifted by the change at the adjacent
    node, O~_0 = O*_0 + (O~_1 - O*_1) (likewise at x = 1), so that the wall cell keeps the
    prediction's net flux and the wall supplies what the corrected interior node draws.
    Eq. bc-pre applied to O~ with the frozen E* would tie the wall inflow to O~_1 with
    the opposite sign (the inflow falls as the interior draws more), which empties a
    cold wall cell or freezes a hot one at the configured dt = dx/2 of the 128-cell
    Marshak slab."""
    if P.kind == SIGMA_CONST:
        return flux_div(P, Os)
    N, M = P.N, P.M
    eps, c, dt, dx = P.eps, P.c, P.dt, P.dx
    V = np.maximum(Us, 0.0) ** (P.p / 4.0)
    Vn = np.zeros(N + 1)
    Vn[1:-1] = 0.5 * (V[:-1] + V[1:])
    sn = P.node_sig()
    d = np.zeros(N + 1)
    den = Vn[1:-1] * eps ** 2 / (c * dt) + sn[1:-1]
    d[1:-1] = np.where(den > 0, Vn[1:-1] / np.where(den > 0, den, 1.0), 0.0)
    O = np.zeros((N + 1, M))
    O[1:-1] = d[1:-1, None] * (eps ** 2 * S.O[1:-1] / (c * dt) - P.v[None, :] * (Es[1:] - Es[:-1]) / dx)
    if P.bc == "inflow":
        O[0] = Os[0] + (O[1] - Os[1])
        O[N] = Os[N] + (O[N - 1] - Os[N - 1])
    return flux_div(P, O)


def step(P, S, info=None):
    """One step of Algorithm 2: prediction, correction (substeps 1 and 2), projection
    (Eq. dis-proj).  Returns the new State; fills `info` if given."""
    Es, Os, Us, _ = predict(P, S)
    Fs = flux_div(P, Os)
    Fc = correction_flux(P, S, Es, Os, Us)
    Tn, its, nneg, rho_n = correction_temperature(P, S, Fc, Us)
    EJ, OJ = correct_intensity(P, S, Tn)
    U = Tn ** 4                                   # Eq. dis-proj1
    E = P.a * P.c * U[:, None] + P.eps * EJ       # Eq. dis-proj3
    O = OJ                                        # Eq. dis-proj2 and its boundary rows
    if info is not None:
        info.Estar, info.Ostar, info.Ustar, info.Fstar = Es, Os, Us, Fs
        info.extra["Fcorr"] = Fc
        info.rho_n, info.T_new, info.newton_its, info.EJ = rho_n, Tn, its, EJ
        info.negative_R = nneg
    return State(E=E, O=O, U=U, T=Tn, t=S.t + P.dt, step=S.step + 1)


def run(P, S, nsteps):
    for _ in range(nsteps):
        S = step(P, S)
    return S


def intensity(P, S):
    """Cell-centre I(+v_k), I(-v_k): E +- eps * (O_j + O_{j+1})/2."""
    Oc = 0.5 * (S.O[:-1] + S.O[1:])
    return S.E + P.eps * Oc, S.E - P.eps * Oc


def energy(P, S):
    """Total energy sum_j dx [rho_j / c + Cv T_j] (Eq. energybalance integrated)."""
    return P.dx * np.sum(rho_of(P, S.E) / P.c + P.Cv * S.T)
