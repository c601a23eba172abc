"""Pins of the 2D oracle (oracle/grte2d.py) against what the paper and the mathematics
fix: the 1D scheme it must reduce to, equilibrium, conservation, the literal system,
the S8 moment conditions, and the exactness of the directional differences on
polynomials (which the 1D reduction cannot see: the mixed mu-eta terms)."""
import numpy as np
import pytest

from oracle import grte1d as o1
from oracle import grte2d as o2
from oracle.quadrature import gauss_legendre_half, level_symmetric_s8, s8_pairs_2d


def test_s8_moments_and_pairs():
    d, w = level_symmetric_s8()
    assert d.shape == (80, 3)
    assert np.allclose(np.sum(d ** 2, axis=1), 1.0, rtol=0, atol=1e-15)
    for comp in range(3):
        x = d[:, comp]
        assert abs(np.sum(w) - 1.0) < 1e-15
        assert abs(np.sum(w * x ** 2) - 1.0 / 3.0) < 1e-15
        assert abs(np.sum(w * x ** 4) - 1.0 / 5.0) < 1e-15
        assert abs(np.sum(w * x ** 6) - 1.0 / 7.0) < 1e-15
        assert abs(np.sum(w * x)) < 1e-15 and abs(np.sum(w * x ** 3)) < 1e-15
    assert len(set(np.round(w, 14))) == 3 and np.all(w > 0)
    mu, eta, wp = s8_pairs_2d()
    assert mu.size == 20 and np.all(mu > 0)
    assert abs(np.sum(wp) - 1.0) < 1e-15
    assert abs(np.sum(wp * mu ** 2) - 1.0 / 3.0) < 1e-15
    assert abs(np.sum(wp * eta ** 2) - 1.0 / 3.0) < 1e-15
    assert abs(np.sum(wp * mu * eta)) < 1e-15


def _profile_problem(axis, kind, eps, n=24, m=3, n_dir=8):
    """A 2D problem that varies only along `axis` (periodic across it) and the 1D
    problem it must reproduce, with the same seeded data."""
    v, w = gauss_legendre_half(n_dir)
    rng = np.random.default_rng(7)
    sig1 = 0.5 + 2.0 * rng.random(n)
    T1 = 0.3 + 0.7 * rng.random(n)
    other = 0.9 - 0.17 * np.arange(v.size)      # the other cosine: arbitrary, nonzero
    dt = 0.4 / n
    P1 = o1.Problem(N=n, v=v, w=w, sig=sig1, eps=eps, dt=dt, kind=kind, bc="inflow",
                    bL=np.full(v.size, 1.0), bR=np.full(v.size, 0.3))
    if axis == "x":
        P2 = o2.Problem2D(Nx=n, Ny=m, mu=v, eta=other, w=w, sig=np.tile(sig1, (m, 1)), eps=eps, dt=dt,
                          kind=kind, bcx="inflow", bcy="periodic", bx0=1.0, bx1=0.3)
        T2 = np.tile(T1, (m, 1))
    else:
        P2 = o2.Problem2D(Nx=m, Ny=n, mu=other, eta=v, w=w, sig=np.tile(sig1[:, None], (1, m)), eps=eps,
                          dt=dt, kind=kind, bcx="periodic", bcy="inflow", by0=1.0, by1=0.3, Lx=1.0, Ly=1.0)
        T2 = np.tile(T1[:, None], (1, m))
    return P1, P2, T1, T2


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("kind,eps", [("const", 1.0), ("const", 1e-2), ("t3", 1e-3)])
def test_reduces_to_1d_scheme(axis, kind, eps):
    P1, P2, T1, T2 = _profile_problem(axis, kind, eps)
    S1 = o1.run(P1, o1.equilibrium_state(P1, T1), 2)
    S2 = o2.run(P2, o2.equilibrium_state(P2, T2.ravel()), 2)
    n, m = P1.N, 3
    if axis == "x":
        T2r = S2.T.reshape(m, n)
        E2r = S2.E.reshape(m, n, -1)
        O2r = S2.O.reshape(m + 1, n + 1, -1)
    else:
        T2r = S2.T.reshape(n, m).T
        E2r = S2.E.reshape(n, m, -1).transpose(1, 0, 2)
        O2r = S2.O.reshape(n + 1, m + 1, -1).transpose(1, 0, 2)
    scaleE = np.abs(S1.E) + eps * np.abs(S1.O[:-1]) + 1e-300
    for r in range(m):
        assert np.max(np.abs(T2r[r] - S1.T) / S1.T) < 1e-12
        assert np.max(np.abs(E2r[r] - S1.E) / scaleE) < 1e-12
    for r in range(m + 1):
        assert np.max(np.abs(O2r[r] - S1.O)) <= 1e-11 * np.max(np.abs(S1.O)) * max(1.0, 1.0 / eps)


@pytest.mark.parametrize("kind", ["const", "t3"])
def test_equilibrium_preserved_with_walls_and_corners(kind):
    mu, eta, w = s8_pairs_2d()
    T = 0.7
    b = T ** 4
    rng = np.random.default_rng(3)
    P = o2.Problem2D(Nx=6, Ny=5, mu=mu, eta=eta, w=w, sig=0.5 + rng.random((5, 6)), eps=1e-3, dt=0.05,
                     kind=kind, bx0=b, bx1=b, by0=b, by1=b)
    S0 = o2.equilibrium_state(P, np.full(P.nc, T))
    S = o2.run(P, S0, 2)
    # rounding at the walls is amplified by 2/eps (the same bound as the 1D pin)
    tol = 1e-14 + 5e-16 / P.eps
    assert np.max(np.abs(S.T - T)) < tol * T
    assert np.max(np.abs(S.E - b)) < tol * b
    assert np.max(np.abs(P.eps * S.O)) < tol * b


def _random_state(P, rng):
    T = 0.4 + 0.6 * rng.random(P.nc)
    E = (T ** 4)[:, None] * (1.0 + 0.2 * rng.random((P.nc, P.K)))
    O = 0.1 * (rng.random((P.nv, P.K)) - 0.5)
    if P.bcx == "periodic":
        O.reshape(P.Ny + 1, P.Nx + 1, P.K)[:, P.Nx] = O.reshape(P.Ny + 1, P.Nx + 1, P.K)[:, 0]
    if P.bcy == "periodic":
        O.reshape(P.Ny + 1, P.Nx + 1, P.K)[P.Ny] = O.reshape(P.Ny + 1, P.Nx + 1, P.K)[0]
    return o2.State2D(E=E, O=O, U=T ** 4, T=T)


@pytest.mark.parametrize("eps", [1.0, 1e-2])
def test_energy_conserved_periodic_uniform_sigma(eps):
    mu, eta, w = s8_pairs_2d()
    P = o2.Problem2D(Nx=7, Ny=6, mu=mu, eta=eta, w=w, sig=1.3, eps=eps, dt=0.03, kind="const",
                     bcx="periodic", bcy="periodic")
    S = _random_state(P, np.random.default_rng(11))
    e0 = o2.energy(P, S)
    for _ in range(3):
        S = o2.step(P, S)
        assert abs(o2.energy(P, S) - e0) < 1e-13 * e0


@pytest.mark.parametrize("eps", [1.0, 0.1])
def test_eliminated_prediction_matches_literal_system(eps):
    mu, eta, w = s8_pairs_2d()
    rng = np.random.default_rng(5)
    P = o2.Problem2D(Nx=6, Ny=5, mu=mu, eta=eta, w=w, sig=0.3 + rng.random((5, 6)), eps=eps, dt=0.04,
                     kind="t3", bx0=1.0, bx1=0.2, by0=0.5, by1=0.0)
    S = _random_state(P, rng)
    E, O, U, _ = o2.predict(P, S)
    El, Ol, Ul = o2.predict_literal(P, S)
    assert np.max(np.abs(E - El)) < 1e-12 * np.max(np.abs(El))
    assert np.max(np.abs(O - Ol)) < 1e-11 * np.max(np.abs(Ol))
    assert np.max(np.abs(U - Ul) / Ul) < 1e-12


def _centres_and_vertices(P):
    xc, yc = np.meshgrid((np.arange(P.Nx) + 0.5) * P.dx, (np.arange(P.Ny) + 0.5) * P.dy)
    xv, yv = np.meshgrid(np.arange(P.Nx + 1) * P.dx, np.arange(P.Ny + 1) * P.dy)
    return xc.ravel(), yc.ravel(), xv.ravel(), yv.ravel()


def test_directional_differences_exact_on_polynomials():
    # The vertex gradient D_k and the cell divergence D*_k are the directional derivative
    # Omega_k . grad, exact on linear fields; through both, quadratics give the second
    # directional derivative exactly: mu^2 f_xx + 2 mu eta f_xy + eta^2 f_yy.  xy pins the
    # sign of the cross terms and which cosine goes with which axis; dx != dy pins the
    # spacings.
    mu, eta, w = s8_pairs_2d()
    P = o2.Problem2D(Nx=7, Ny=5, mu=mu, eta=eta, w=w, sig=1.0, Lx=1.3, Ly=0.7)
    xc, yc, xv, yv = _centres_and_vertices(P)
    vi, vj = np.arange(P.nv) % (P.Nx + 1), np.arange(P.nv) // (P.Nx + 1)
    node = (vi > 0) & (vi < P.Nx) & (vj > 0) & (vj < P.Ny)          # vertices with a node equation
    cp, cq = np.arange(P.nc) % P.Nx, np.arange(P.nc) // P.Nx
    inner = (cp > 0) & (cp < P.Nx - 1) & (cq > 0) & (cq < P.Ny - 1)   # cells whose 4 vertices are nodes
    for k in range(P.K):
        Dk, Ds = o2.grad_matrix(P, k), o2.div_matrix(P, k)
        m, e = mu[k], eta[k]
        for a, b in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.9)):
            g = Dk @ (a * xc + b * yc + 0.3)
            assert np.allclose(g[node], m * a + e * b, rtol=0, atol=1e-12)
            assert np.all(g[~node] == 0.0)
            d = Ds @ (a * xv + b * yv - 0.2)
            assert np.allclose(d, m * a + e * b, rtol=0, atol=1e-12)
        for f, want in ((xc ** 2, 2 * m * m), (xc * yc, 2 * m * e), (yc ** 2, 2 * e * e)):
            second = Ds @ (Dk @ f)
            assert np.allclose(second[inner], want, rtol=0, atol=1e-11), (k, want)


@pytest.mark.parametrize("kind", ["const", "t3"])
def test_reflection_and_transpose_symmetry(kind):
    # The S8 pair set is symmetric under x -> -x and under x <-> y, so a problem with
    # data symmetric under the reflection x -> Lx - x (or, on a square grid, under the
    # transpose) keeps that symmetry step by step; a wall treatment that favours one
    # side or one axis breaks it.
    mu, eta, w = s8_pairs_2d()
    n = 6
    rng = np.random.default_rng(41)
    base = 0.5 + rng.random((n, n))
    sig = base + base[:, ::-1] + base.T + base.T[:, ::-1]          # symmetric both ways
    sig = sig + sig[::-1, :]
    T = 0.3 + 0.2 * rng.random((n, n))
    T = T + T[:, ::-1] + T.T + T.T[:, ::-1]
    T = 0.25 * (T + T[::-1, :]) / 2.0
    P = o2.Problem2D(Nx=n, Ny=n, mu=mu, eta=eta, w=w, sig=sig, eps=1e-2, dt=0.02, kind=kind,
                     bx0=0.8, bx1=0.8, by0=0.8, by1=0.8)
    S = o2.equilibrium_state(P, T.ravel())
    for _ in range(2):
        S = o2.step(P, S)
        Tn = S.T.reshape(n, n)
        assert np.max(np.abs(Tn - Tn[:, ::-1])) < 1e-12 * np.max(Tn)      # x -> Lx - x
        assert np.max(np.abs(Tn - Tn.T)) < 1e-12 * np.max(Tn)             # x <-> y
