"""2D fully discrete AP scheme for the gray radiative transfer equation (oracle).

TEST INFRASTRUCTURE ONLY - see oracle/__init__.py.

The paper derives the scheme in 1D (Algorithm 2, Sec. 4; sigma/T^3 form, Sec. 5)
and states that it extends to several dimensions direction by direction (Sec. 4,
first paragraph) without writing the 2D form; this module is the reading used here
(reading Q17), built so that it reduces exactly to the 1D scheme of grte1d for data
that do not depend on y (or on x):

  cells    (p, q), p = 0..Nx-1, q = 0..Ny-1, centre ((p+1/2) dx, (q+1/2) dy): E, U, T
  vertices (i, j), i = 0..Nx,   j = 0..Ny,   at (i dx, j dy): O
  pairs    k = 0..K-1 of directions Omega_k = (mu_k, eta_k) and -Omega_k, weights
           w_k with sum_k w_k = 1; E = (I(Omega) + I(-Omega))/2,
           O = (I(Omega) - I(-Omega))/(2 eps)  (Eq. EO in each pair).

Vertex (i, j) touches the cells (i-1, j-1), (i, j-1), (i-1, j), (i, j).  The
streaming derivative of E at a vertex averages the two cell differences across it:

  (D_k E)_ij = mu_k [E(i,j-1) + E(i,j) - E(i-1,j-1) - E(i-1,j)] / (2 dx)
             + eta_k [E(i-1,j) + E(i,j) - E(i-1,j-1) - E(i,j-1)] / (2 dy)

and the streaming derivative of O at a cell averages the two vertex differences
along each side:

  (D*_k O)_pq = mu_k [O(p+1,q) + O(p+1,q+1) - O(p,q) - O(p,q+1)] / (2 dx)
              + eta_k [O(p,q+1) + O(p+1,q+1) - O(p,q) - O(p+1,q)] / (2 dy).

With v (E_i - E_{i-1})/dx -> D_k E and v (O_{j+1} - O_j)/dx -> D*_k O the node,
cell and U equations of Eq. dis-pre / Eq. dis-pre-marshak, Eq. Tnp1, Eq. dis-cor /
Eq. dis-cor-marshak and Eq. dis-proj are taken over unchanged.  Vertex opacity is the
harmonic mean of the four cells, vertex kappa (sigma/T^3) their mean.

Boundaries, per axis: 'periodic' (vertex Nx is vertex 0, cell -1 is cell Nx-1), or
'inflow' with an isotropic inflow intensity per side (b = 0: vacuum).  A cell beside
an inflow wall applies Eq. bc-pre to its own wall side, exactly as the 1D wall cell:
the mean of O over that side obeys
  side = 2/eps (b - E_cell) - opposite side      (Omega_k enters the domain there)
  side = 2/eps (E_cell - b) - opposite side      (-Omega_k enters)
(div_operator).  An inflow wall vertex itself (needed for the opposite side of a
corner cell and for the output) uses the same relation along the wall normal with E
the mean of the two wall cells beside it and the next vertex inward; a corner vertex
takes the mean of its two walls' values (E_wall = the corner cell).  Applying the
wall relation per cell rather than per vertex keeps a cell's outflow from depending
on its neighbours' E along the wall (with the vertex form, a cold wall cell beside a
hot one was drained by its neighbour's outflow).

Parity unpinned: the value of O at the four corner vertices of a grid with two inflow
walls (the corner mean above).  No cell's update reads it, so it reaches only the
reported O there, and no invariant or limit fixes it.

Linear solves (sparse LU throughout): the prediction on the unknowns (e, rho) with
E = rho + e exactly as grte1d.coefficients() (O eliminated by the vertex map
O_k = Q_k E_k + q_k, U* by Eq. dis-pre3); predict_literal() assembles the unknowns
(E, O, U) literally as a check.  Correction substep 2 solves, per pair,
(A + G_k) E_J = rhs with E = a c U + eps E_J.
"""
from dataclasses import dataclass
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .scalar import quartic_root

SIGMA_CONST = "const"
SIGMA_T3 = "t3"


@dataclass
class Problem2D:
    Nx: int
    Ny: int
    mu: np.ndarray           # (K,)
    eta: np.ndarray          # (K,)
    w: np.ndarray            # (K,), sum = 1
    sig: np.ndarray          # (Ny, Nx) sigma(x) or sigma_0(x) per cell
    a: float = 1.0
    c: float = 1.0
    Cv: float = 1.0
    eps: float = 1.0
    dt: float = 1e-3
    kind: str = SIGMA_CONST
    bcx: str = "inflow"      # 'inflow' or 'periodic'
    bcy: str = "inflow"
    bx0: float = 0.0         # isotropic inflow intensity on x = x0, x1, y = y0, y1
    bx1: float = 0.0
    by0: float = 0.0
    by1: float = 0.0
    Lx: float = 1.0
    Ly: float = 1.0
    p: float = 3.0           # the exponent of sigma_0/T^p (kind 't3'; see grte1d)

    def __post_init__(self):
        self.mu = np.asarray(self.mu, dtype=np.float64)
        self.eta = np.asarray(self.eta, dtype=np.float64)
        self.w = np.asarray(self.w, dtype=np.float64)
        self.sig = np.broadcast_to(np.asarray(self.sig, dtype=np.float64), (self.Ny, self.Nx)).copy()

    @property
    def K(self):
        return self.mu.size

    @property
    def dx(self):
        return self.Lx / self.Nx

    @property
    def dy(self):
        return self.Ly / self.Ny

    @property
    def nc(self):
        return self.Nx * self.Ny

    @property
    def nv(self):
        return (self.Nx + 1) * (self.Ny + 1)

    def cell(self, p, q):
        """Flat cell index, wrapping periodic axes; None outside the domain."""
        if self.bcx == "periodic":
            p %= self.Nx
        if self.bcy == "periodic":
            q %= self.Ny
        if 0 <= p < self.Nx and 0 <= q < self.Ny:
            return q * self.Nx + p
        return None

    def vert(self, i, j):
        return j * (self.Nx + 1) + i


@dataclass
class State2D:
    E: np.ndarray   # (nc, K)
    O: np.ndarray   # (nv, K)
    U: np.ndarray   # (nc,)
    T: np.ndarray   # (nc,)


def equilibrium_state(P, T):
    """I = a c T^4: E = a c T^4, O = 0, U = T^4 (Q10)."""
    T = np.broadcast_to(np.asarray(T, dtype=np.float64).ravel(), (P.nc,)).copy()
    U = T ** 4
    return State2D(E=np.repeat((P.a * P.c * U)[:, None], P.K, axis=1), O=np.zeros((P.nv, P.K)), U=U, T=T)


def rho_of(P, E):
    return E @ P.w


def _kappa_theta(P, T):
    if P.kind == SIGMA_CONST:
        return np.ones(P.nc), T ** 3
    return T ** P.p, T ** (3.0 - P.p)


def _vertex_kind(P, i, j):
    """'interior' (node equation), 'x', 'y' (one inflow wall) or 'corner'."""
    onx = P.bcx == "inflow" and i in (0, P.Nx)
    ony = P.bcy == "inflow" and j in (0, P.Ny)
    if onx and ony:
        return "corner"
    if onx:
        return "x"
    if ony:
        return "y"
    if (P.bcx == "periodic" and i == P.Nx) or (P.bcy == "periodic" and j == P.Ny):
        return "copy"
    return "interior"


def _vertex_cells(P, i, j):
    return (P.cell(i - 1, j - 1), P.cell(i, j - 1), P.cell(i - 1, j), P.cell(i, j))


def _vertex_coef(P, kc):
    """kappa and sigma (harmonic mean) at the vertices that carry a node equation."""
    kv = np.zeros(P.nv)
    sv = np.zeros(P.nv)
    sg = P.sig.ravel()
    for j in range(P.Ny + 1):
        for i in range(P.Nx + 1):
            if _vertex_kind(P, i, j) != "interior":
                continue
            cs = _vertex_cells(P, i, j)
            v = P.vert(i, j)
            kv[v] = np.mean([kc[c] for c in cs])
            s = np.array([sg[c] for c in cs])
            sv[v] = 4.0 / np.sum(1.0 / s) if np.all(s > 0) else 0.0
    return kv, sv


def grad_matrix(P, k):
    """D_k: cells -> vertices (rows of vertices with a node equation only)."""
    rows, cols, vals = [], [], []
    mu, eta = P.mu[k], P.eta[k]
    for j in range(P.Ny + 1):
        for i in range(P.Nx + 1):
            if _vertex_kind(P, i, j) != "interior":
                continue
            c00, c10, c01, c11 = _vertex_cells(P, i, j)
            v = P.vert(i, j)
            for cidx, val in ((c10, mu / (2 * P.dx)), (c11, mu / (2 * P.dx)), (c00, -mu / (2 * P.dx)),
                              (c01, -mu / (2 * P.dx)), (c01, eta / (2 * P.dy)), (c11, eta / (2 * P.dy)),
                              (c00, -eta / (2 * P.dy)), (c10, -eta / (2 * P.dy))):
                rows.append(v)
                cols.append(cidx)
                vals.append(val)
    return sp.csr_matrix((vals, (rows, cols)), shape=(P.nv, P.nc))


def div_matrix(P, k):
    """D*_k: vertices -> cells, without wall rows (the plain 2x2 side averages)."""
    rows, cols, vals = [], [], []
    mu, eta = P.mu[k], P.eta[k]
    for q in range(P.Ny):
        for p in range(P.Nx):
            c = q * P.Nx + p
            v00, v10, v01, v11 = P.vert(p, q), P.vert(p + 1, q), P.vert(p, q + 1), P.vert(p + 1, q + 1)
            for vidx, val in ((v10, mu / (2 * P.dx)), (v11, mu / (2 * P.dx)), (v00, -mu / (2 * P.dx)),
                              (v01, -mu / (2 * P.dx)), (v01, eta / (2 * P.dy)), (v11, eta / (2 * P.dy)),
                              (v00, -eta / (2 * P.dy)), (v10, -eta / (2 * P.dy))):
                rows.append(c)
                cols.append(vidx)
                vals.append(val)
    return sp.csr_matrix((vals, (rows, cols)), shape=(P.nc, P.nv))


def div_operator(P, k):
    """The streaming derivative of O at the cells as used by the scheme:
    (D*_k O)_c + ed_c E_c + bt_c.  A cell beside an inflow wall takes its wall side
    from Eq. bc-pre with its own E, as the 1D wall cell does: for the x = 0 side
    (mean of its two wall vertices, L) with R the opposite side's mean,
      L = s 2/eps (b - E_c) - R,  so  mu (R - L)/dx = mu (2 R - s 2/eps (b - E_c))/dx,
    and likewise on the other walls.  Returns (D (nc x nv), ed (nc,), bt (nc,))."""
    rows, cols, vals = [], [], []
    ed = np.zeros(P.nc)
    bt = np.zeros(P.nc)
    mu, eta = P.mu[k], P.eta[k]
    for q in range(P.Ny):
        for p in range(P.Nx):
            c = q * P.Nx + p
            v00, v10, v01, v11 = P.vert(p, q), P.vert(p + 1, q), P.vert(p, q + 1), P.vert(p + 1, q + 1)
            # side weights (L, R along x; B, T along y) of mu/dx and eta/dy
            wL, wR, wB, wT = -1.0, 1.0, -1.0, 1.0
            for axis, comp, h_, side_lo, side_hi in (("x", mu, P.dx, p == 0, p == P.Nx - 1),
                                                       ("y", eta, P.dy, q == 0, q == P.Ny - 1)):
                inflow = (P.bcx if axis == "x" else P.bcy) == "inflow"
                if not inflow:
                    continue
                if side_lo:      # low side replaced: comp (2 hi - s 2/eps (b - E))/h
                    s_, b = _wall(P, k, axis, 0)
                    if axis == "x":
                        wL, wR = 0.0, 2.0
                    else:
                        wB, wT = 0.0, 2.0
                    ed[c] += comp * s_ * 2.0 / P.eps / h_
                    bt[c] -= comp * s_ * 2.0 / P.eps * b / h_
                if side_hi:      # high side replaced: comp (s 2/eps (b - E) - 2 lo)/h
                    s_, b = _wall(P, k, axis, 1)
                    if axis == "x":
                        wL, wR = (wL if side_lo else -2.0), 0.0
                    else:
                        wB, wT = (wB if side_lo else -2.0), 0.0
                    ed[c] -= comp * s_ * 2.0 / P.eps / h_
                    bt[c] += comp * s_ * 2.0 / P.eps * b / h_
            for vidx, val in ((v00, wL * mu / (2 * P.dx)), (v01, wL * mu / (2 * P.dx)),
                              (v10, wR * mu / (2 * P.dx)), (v11, wR * mu / (2 * P.dx)),
                              (v00, wB * eta / (2 * P.dy)), (v10, wB * eta / (2 * P.dy)),
                              (v01, wT * eta / (2 * P.dy)), (v11, wT * eta / (2 * P.dy))):
                if val != 0.0:
                    rows.append(c)
                    cols.append(vidx)
                    vals.append(val)
    return sp.csr_matrix((vals, (rows, cols)), shape=(P.nc, P.nv)), ed, bt


def _wall(P, k, axis, side):
    """(s, b): O = s * 2/eps (b - E_wall) - O_inner with s = +1 if Omega_k enters the
    domain through this wall, else s = -1 (then -Omega_k enters and O = 2/eps
    (E_wall - b) - O_inner)."""
    comp = P.mu[k] if axis == "x" else P.eta[k]
    if comp == 0.0:
        raise ValueError("a direction parallel to an inflow wall")
    enters = comp > 0 if side == 0 else comp < 0
    b = {("x", 0): P.bx0, ("x", 1): P.bx1, ("y", 0): P.by0, ("y", 1): P.by1}[(axis, side)]
    return (1.0 if enters else -1.0), b


def vertex_map(P, k, E_coef, o):
    """O_k = Q E_k + q for pair k, from the node equation O = o - d D_k E (interior
    vertices, E_coef = diag(d) D_k), the wall expressions and the corner means.
    o: (nv,) data part d eps^2 O^n/(c dt) of the interior vertices."""
    nv, nc = P.nv, P.nc
    Q = sp.lil_matrix((nv, nc))
    q = np.zeros(nv)
    Ei = (-E_coef).tolil()
    for v in range(nv):
        Q.rows[v] = list(Ei.rows[v])
        Q.data[v] = list(Ei.data[v])
    q[:] = o
    Q = Q.tocsr()
    rowsQ = {v: Q.getrow(v) for v in range(nv)}

    def wall_expr(i, j, axis):
        side = 0 if (i == 0 if axis == "x" else j == 0) else 1
        s, b = _wall(P, k, axis, side)
        if axis == "x":
            ii = 1 if i == 0 else P.Nx - 1
            inner = P.vert(ii, j)
            cells = [c for c in (P.cell(0 if i == 0 else P.Nx - 1, j - 1), P.cell(0 if i == 0 else P.Nx - 1, j))
                     if c is not None]
        else:
            jj = 1 if j == 0 else P.Ny - 1
            inner = P.vert(i, jj)
            cells = [c for c in (P.cell(i - 1, 0 if j == 0 else P.Ny - 1), P.cell(i, 0 if j == 0 else P.Ny - 1))
                     if c is not None]
        row = sp.csr_matrix((np.full(len(cells), -s * 2.0 / P.eps / len(cells)), ([0] * len(cells), cells)),
                            shape=(1, nc))
        return row - rowsQ[inner], s * 2.0 / P.eps * b - q[inner]

    order = {"interior": 0, "copy": 1, "x": 2, "y": 2, "corner": 3}
    verts = sorted(((order[_vertex_kind(P, i, j)], i, j) for j in range(P.Ny + 1) for i in range(P.Nx + 1)))
    for _, i, j in verts:
        kind = _vertex_kind(P, i, j)
        v = P.vert(i, j)
        if kind == "interior":
            continue
        if kind == "copy":
            src = P.vert(i % P.Nx if P.bcx == "periodic" else i, j % P.Ny if P.bcy == "periodic" else j)
            rowsQ[v], q[v] = rowsQ[src], q[src]
        elif kind in ("x", "y"):
            rowsQ[v], q[v] = wall_expr(i, j, kind)
        else:
            rx, qx = wall_expr(i, j, "x")
            ry, qy = wall_expr(i, j, "y")
            rowsQ[v], q[v] = 0.5 * (rx + ry), 0.5 * (qx + qy)
    Q = sp.vstack([rowsQ[v] for v in range(nv)]).tocsr()
    return Q, q


def coefficients(P, T, Oold):
    """Per-cell coefficients at temperature T and, per pair, the eliminated streaming
    operator G_k = diag(kappa) (D*_k Q_k + diag(ed_k)), its data part
    phi_k = kappa (D*_k q_k + bt_k) (div_operator) and the vertex map (Q_k, q_k)
    (names as grte1d.coefficients)."""
    eps, c, a, dt, Cv = P.eps, P.c, P.a, P.dt, P.Cv
    kc, theta = _kappa_theta(P, T)
    sc = P.sig.ravel()
    kv, sv = _vertex_coef(P, kc)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(kv > 0, kv / (kv * eps ** 2 / (c * dt) + sv), 0.0)
    s = sc * Cv / (Cv * eps ** 2 + 4.0 * sc * theta * dt * a * c)
    gam = 4.0 * sc * theta * dt / (eps ** 2 * Cv)
    ops = []
    for k in range(P.K):
        Dk = grad_matrix(P, k)
        Dsk, ed, bt = div_operator(P, k)
        o = d * eps ** 2 / (c * dt) * Oold[:, k]
        Qk, qk = vertex_map(P, k, sp.diags(d) @ Dk, o)
        Gk = sp.diags(kc) @ (Dsk @ Qk + sp.diags(ed))
        phik = kc * (Dsk @ qk + bt)
        ops.append(dict(G=Gk.tocsr(), phi=phik, Q=Qk, q=qk, Ds=Dsk, ed=ed, bt=bt))
    return dict(kc=kc, theta=theta, s=s, gam=gam, d=d, A=kc / (c * dt) + sc / eps ** 2,
                alpha=kc / (c * dt) + s, ops=ops)


def predict(P, S):
    """Prediction solved exactly on (e, rho) (see grte1d.coefficients()):
      A e_k + G_k (rho + e_k) + phi_k = kappa (E^n_k - rho)/(c dt) - s (rho - a c U^n)
      alpha rho + sum_k w_k [G_k (rho + e_k) + phi_k] = kappa rho^n/(c dt) + s a c U^n.
    Returns (E*, O*, U*, rho*)."""
    K, nc = P.K, P.nc
    c, a, dt = P.c, P.a, P.dt
    C = coefficients(P, S.T, S.O)
    rho_n = S.E @ P.w
    A = sp.diags(C["A"])
    al = sp.diags(C["alpha"])
    blocks = [[None] * (K + 1) for _ in range(K + 1)]
    rhs = np.zeros((K + 1) * nc)
    Gsum = sp.csr_matrix((nc, nc))
    phisum = np.zeros(nc)
    for k, op in enumerate(C["ops"]):
        G = op["G"]
        blocks[k][k] = A + G
        blocks[k][K] = G + al
        blocks[K][k] = P.w[k] * G
        Gsum = Gsum + P.w[k] * G
        phisum += P.w[k] * op["phi"]
        rhs[k * nc:(k + 1) * nc] = C["kc"] * S.E[:, k] / (c * dt) + C["s"] * a * c * S.U - op["phi"]
    blocks[K][K] = al + Gsum
    rhs[K * nc:] = C["kc"] * rho_n / (c * dt) + C["s"] * a * c * S.U - phisum
    M = sp.bmat(blocks, format="csc")
    z = spla.spsolve(M, rhs)
    rho = z[K * nc:]
    e = z[:K * nc].reshape(K, nc).T
    E = rho[:, None] + e
    O = np.zeros((P.nv, K))
    for k, op in enumerate(C["ops"]):
        O[:, k] = op["Q"] @ E[:, k] + op["q"]
    U = (S.U + C["gam"] * rho) / (1.0 + C["gam"] * a * c)
    return E, O, U, rho


def predict_literal(P, S):
    """The prediction assembled literally in (E, O, U) and solved by sparse LU
    (accurate while eps is not small); an independent check of predict()."""
    K, nc, nv = P.K, P.nc, P.nv
    eps, c, a, dt, Cv = P.eps, P.c, P.a, P.dt, P.Cv
    kc, theta = _kappa_theta(P, S.T)
    kv, sv = _vertex_coef(P, kc)
    sc = P.sig.ravel()
    nE, nO = K * nc, K * nv
    n = nE + nO + nc
    rows, cols, vals = [], [], []
    b = np.zeros(n)

    def add(r, ci, val):
        rows.append(r)
        cols.append(ci)
        vals.append(val)

    iE = lambda cc, k: k * nc + cc
    iO = lambda v, k: nE + k * nv + v
    iU = lambda cc: nE + nO + cc
    for k in range(K):
        Dsm, ed, bt = div_operator(P, k)
        Ds = Dsm.tocoo()
        for cc in range(nc):
            add(iE(cc, k), iE(cc, k), kc[cc] / (c * dt) + sc[cc] / eps ** 2 + kc[cc] * ed[cc])
            add(iE(cc, k), iU(cc), -sc[cc] * a * c / eps ** 2)
            b[iE(cc, k)] = kc[cc] * S.E[cc, k] / (c * dt) - kc[cc] * bt[cc]
        for r, v, val in zip(Ds.row, Ds.col, Ds.data):
            add(iE(r, k), iO(v, k), kc[r] * val)
        Dk = grad_matrix(P, k).tocoo()
        for r, cc, val in zip(Dk.row, Dk.col, Dk.data):
            add(iO(r, k), iE(cc, k), kv[r] * val / eps ** 2)
        for j in range(P.Ny + 1):
            for i in range(P.Nx + 1):
                v = P.vert(i, j)
                kind = _vertex_kind(P, i, j)
                r = iO(v, k)
                if kind == "interior":
                    add(r, r, kv[v] / (c * dt) + sv[v] / eps ** 2)
                    b[r] = kv[v] * S.O[v, k] / (c * dt)
                elif kind == "copy":
                    src = P.vert(i % P.Nx if P.bcx == "periodic" else i, j % P.Ny if P.bcy == "periodic" else j)
                    add(r, r, 1.0)
                    add(r, iO(src, k), -1.0)
                else:
                    axes = ["x", "y"] if kind == "corner" else [kind]
                    f = 1.0 / len(axes)
                    add(r, r, 1.0)
                    for ax in axes:
                        side = 0 if (i == 0 if ax == "x" else j == 0) else 1
                        s_, bb = _wall(P, k, ax, side)
                        if ax == "x":
                            inner = P.vert(1 if i == 0 else P.Nx - 1, j)
                            cells = [cc for cc in (P.cell(0 if i == 0 else P.Nx - 1, j - 1),
                                                   P.cell(0 if i == 0 else P.Nx - 1, j)) if cc is not None]
                        else:
                            inner = P.vert(i, 1 if j == 0 else P.Ny - 1)
                            cells = [cc for cc in (P.cell(i - 1, 0 if j == 0 else P.Ny - 1),
                                                   P.cell(i, 0 if j == 0 else P.Ny - 1)) if cc is not None]
                        add(r, iO(inner, k), f)
                        for cc in cells:
                            add(r, iE(cc, k), f * s_ * 2.0 / eps / len(cells))
                        b[r] += f * s_ * 2.0 / eps * bb
    for cc in range(nc):
        g = 4.0 * sc[cc] * theta[cc] / eps ** 2
        add(iU(cc), iU(cc), Cv / dt + g * a * c)
        for k in range(K):
            add(iU(cc), iE(cc, k), -g * P.w[k])
        b[iU(cc)] = Cv * S.U[cc] / dt
    M = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    x = spla.spsolve(M, b)
    E = x[:nE].reshape(K, nc).T
    O = x[nE:nE + nO].reshape(K, nv).T
    U = x[nE + nO:]
    return E, O, U


def flux_div(P, O, E):
    """sum_k w_k (streaming derivative of O_k) per cell (the angular integral of
    Eq. Tnp1, divided by the cell width as in grte1d: Fstar/dx); wall cells through
    div_operator, which needs E."""
    out = np.zeros(P.nc)
    for k in range(P.K):
        Ds, ed, bt = div_operator(P, k)
        out += P.w[k] * (Ds @ O[:, k] + ed * E[:, k] + bt)
    return out


def correction_flux(P, S, Es, Os, Us):
    """The flux the temperature equation of the correction takes from the predicted
    state (see grte1d.correction_flux): sigma(x) the prediction's own O*; sigma/T^3 the
    vertex map rebuilt with the multiplier V* = (U*)^{3/4} (vertex values the mean of
    the four cells) in place of the prediction's K^n, applied to the predicted E*; at
    the inflow-wall vertices the prediction's value plus the change at the inner vertex
    (the reading of grte1d.correction_flux for the walls)."""
    if P.kind == SIGMA_CONST:
        return flux_div(P, Os, Es)
    eps, c, dt = P.eps, P.c, P.dt
    V = np.maximum(Us, 0.0) ** (P.p / 4.0)
    kv, sv = _vertex_coef(P, V)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(kv > 0, kv / (kv * eps ** 2 / (c * dt) + sv), 0.0)
    Oc = np.zeros((P.nv, P.K))
    for k in range(P.K):
        Dk = grad_matrix(P, k)
        o = d * eps ** 2 / (c * dt) * S.O[:, k]
        Qk, qk = vertex_map(P, k, sp.diags(d) @ Dk, o)
        Oc[:, k] = Qk @ Es[:, k] + qk
    # inflow-wall vertices: the prediction's value shifted by the change at the inner
    # vertex (the indices clamped into the interior along the inflow axes), as in 1D
    for j in range(P.Ny + 1):
        for i in range(P.Nx + 1):
            if _vertex_kind(P, i, j) not in ("x", "y", "corner"):
                continue
            ii = min(max(i, 1), P.Nx - 1) if P.bcx == "inflow" else i
            jj = min(max(j, 1), P.Ny - 1) if P.bcy == "inflow" else j
            v, vin = P.vert(i, j), P.vert(ii, jj)
            Oc[v] = Os[v] + (Oc[vin] - Os[vin])
    # a cell beside an inflow wall takes the part of its flux along that wall's normal
    # from the prediction's O* (its wall side is Eq. bc-pre of its own E*, so with the
    # wall value shifted as above the normal part equals the prediction's, as the 1D wall
    # cell's flux does); the part along the wall reads O~
    F = flux_div(P, Oc, Es)
    for k in range(P.K):
        F += P.w[k] * (_wall_normal_operator(P, k) @ (Os[:, k] - Oc[:, k]))
    return F


def _wall_normal_operator(P, k):
    """The vertex terms of div_operator along the normal of each inflow wall, in the
    cells beside that wall (nc x nv); zero elsewhere."""
    rows, cols, vals = [], [], []
    for q in range(P.Ny):
        for p in range(P.Nx):
            c = q * P.Nx + p
            v00, v10, v01, v11 = P.vert(p, q), P.vert(p + 1, q), P.vert(p, q + 1), P.vert(p + 1, q + 1)
            for axis, comp, h_, lo, hi in (("x", P.mu[k], P.dx, p == 0, p == P.Nx - 1),
                                           ("y", P.eta[k], P.dy, q == 0, q == P.Ny - 1)):
                if (P.bcx if axis == "x" else P.bcy) != "inflow" or not (lo or hi):
                    continue
                wlo = 0.0 if lo else -2.0
                whi = 0.0 if hi else 2.0
                if axis == "x":
                    terms = ((v00, wlo), (v01, wlo), (v10, whi), (v11, whi))
                else:
                    terms = ((v00, wlo), (v10, wlo), (v01, whi), (v11, whi))
                for vidx, wgt in terms:
                    if wgt != 0.0:
                        rows.append(c)
                        cols.append(vidx)
                        vals.append(wgt * comp / (2.0 * h_))
    return sp.csr_matrix((vals, (rows, cols)), shape=(P.nc, P.nv))


def correction_temperature(P, S, Fdiv, Ustar):
    """Eq. Tnp1 (sigma/T^3: Eq. dis-cor-marshak4 + 5) multiplied by sig:
    A T^4 + B T = R with R = sig (rho^n/(c dt) - Fdiv) + B T^n (see grte1d)."""
    eps, c, a, dt, Cv = P.eps, P.c, P.a, P.dt, P.Cv
    sig = P.sig.ravel()
    rho_n = rho_of(P, S.E)
    kap = np.ones(P.nc) if P.kind == SIGMA_CONST else np.maximum(Ustar, 0.0) ** (P.p / 4.0)
    A = sig * a / dt
    B = sig * Cv / dt + eps ** 2 * kap * Cv / (c * dt ** 2)
    R = sig * (rho_n / (c * dt) - Fdiv) + B * S.T
    T, its = quartic_root(A, B, R)
    T = np.where(np.isnan(T), S.T, T)
    return T, its, rho_n


def correct_intensity(P, S, Tnew):
    """Correction substep 2 and projection: per pair, with the coefficients at
    T^{n+1} and U = (T^{n+1})^4 (Eq. dis-cor / Eq. dis-cor-marshak, K -> (T^{n+1})^3),
      (A + G_k) E_J = [kappa (E^n_k - a c U)/(c dt) - G_k (a c U) - phi_k] / eps,
    E^{n+1} = a c U + eps E_J (Eq. dis-proj), O^{n+1} = Q_k E^{n+1} + q_k.
    Returns (E_J, E^{n+1}, O^{n+1})."""
    c, a, dt, eps = P.c, P.a, P.dt, P.eps
    U = Tnew ** 4
    C = coefficients(P, Tnew, S.O)
    EJ = np.zeros((P.nc, P.K))
    En = np.zeros((P.nc, P.K))
    On = np.zeros((P.nv, P.K))
    acU = a * c * U
    for k, op in enumerate(C["ops"]):
        M = (sp.diags(C["A"]) + op["G"]).tocsc()
        r = (C["kc"] * (S.E[:, k] - acU) / (c * dt) - op["G"] @ acU - op["phi"]) / eps
        EJ[:, k] = spla.spsolve(M, r)
        En[:, k] = acU + eps * EJ[:, k]
        On[:, k] = op["Q"] @ En[:, k] + op["q"]
    return EJ, En, On


def step(P, S, info=None):
    """One step: prediction, correction substeps 1 and 2, projection."""
    Es, Os, Us, rhos = predict(P, S)
    Fd = flux_div(P, Os, Es)
    Fc = correction_flux(P, S, Es, Os, Us)
    Tn, its, rho_n = correction_temperature(P, S, Fc, Us)
    EJ, En, On = correct_intensity(P, S, Tn)
    if info is not None:
        info.update(Estar=Es, Ostar=Os, Ustar=Us, rho_star=rhos, Fdiv=Fd, Fcorr=Fc, rho_n=rho_n, T_new=Tn,
                    newton_its=its, EJ=EJ)
    return State2D(E=En, O=On, U=Tn ** 4, T=Tn)


def run(P, S, nsteps):
    for _ in range(nsteps):
        S = step(P, S)
    return S


def energy(P, S):
    """sum over cells dx dy [rho/c + Cv T]."""
    return P.dx * P.dy * np.sum(rho_of(P, S.E) / P.c + P.Cv * S.T)
