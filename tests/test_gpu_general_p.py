"""sigma_0/T^p for a general exponent (GRTE_SIGMA_POW) on the GPU against the oracle:
1D FP64 per step to the parity tolerance (inflow and reflecting walls, p = 0.5, 1.5, 2,
and p = 0, which is the sigma(x) scheme), the one-kernel mixed solve to 1e-5, and 2D FP64;
out-of-range p refused."""
import numpy as np
import pytest

from oracle import grte1d as og
from oracle import grte2d as og2
from oracle.quadrature import gauss_legendre_half, s8_pairs_2d
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte
    return grte


def make(G, N, nv, eps, p, bc="inflow", prec=None):
    v, w = gauss_legendre_half(nv)
    sig = 0.5 + 2.0 * wl.SplitMix64(N + nv).uniform(N)
    P = og.Problem(N=N, v=v, w=w, sig=sig, eps=eps, dt=0.5 / N, kind="t3", p=p, bc=bc,
                   bL=np.full(v.size, 0.9), bR=np.full(v.size, 0.1))
    spec = dict(nx=N, n_angle=v.size, v=v, w=w, sigma=sig, kind=G.SIGMA_POW, p=p,
                bc=G.BC_INFLOW if bc == "inflow" else G.BC_REFLECT, bL=P.bL, bR=P.bR, dt=P.dt, eps=eps)
    return P, spec


def state(P, seed):
    rng = wl.SplitMix64(3000 + seed)
    T, E, O = wl.random_state_1d(rng, P.N, P.M, (0.05, 1.0))
    if P.bc == "reflect":
        O[0] = O[-1] = 0.0
    return og.State(E=E, O=O, U=T ** 4, T=T)


@pytest.mark.parametrize("p", [0.0, 0.5, 1.5, 2.0])
@pytest.mark.parametrize("bc", ["inflow", "reflect"])
def test_fp64_one_step_vs_oracle(G, p, bc):
    P, spec = make(G, 96, 8, 1e-2, p, bc)
    S = state(P, int(10 * p))
    h = G.Grte([spec])
    h.set_state(0, S.T, S.E, S.O)
    h.step(1)
    S1 = og.step(P, S)
    tol = np.full(P.N, 1e-12)
    if bc == "inflow":
        tol[0] = tol[-1] = 1e-12 + 4e-15 / P.eps
    err = np.abs(h.T(0, allow=(5,)) - S1.T) / np.maximum(S1.T, 1e-300)
    print("p %.1f %s: T vs oracle %.2e" % (p, bc, err.max()))
    assert np.all(err <= tol)
    h.close()


def test_p0_equals_sigma_x_on_gpu(G):
    P, spec = make(G, 200, 16, 1e-3, 0.0)
    S = state(P, 4)
    h0 = G.Grte([spec])
    hc = G.Grte([dict(spec, kind=G.SIGMA_CONST)])
    for h in (h0, hc):
        h.set_state(0, S.T, S.E, S.O)
        h.step(3)
    a, b = h0.T(0, allow=(5,)), hc.T(0, allow=(5,))
    assert np.max(np.abs(a - b) / b) < 1e-12
    h0.close()
    hc.close()


def test_mixed_one_kernel_solve_p2(G):
    """One step of the one-kernel mixed solve from a smooth state (a cell-by-cell random
    state makes single cells' T ill-conditioned: some nearly empty in the step)."""
    P, spec = make(G, 1500, 16, 1e-2, 2.0)
    T0 = wl.smoothed_log_uniform_T(wl.SplitMix64(77), P.N, 0.1, 1.0, width=9)
    S = og.equilibrium_state(P, T0)
    h = G.Grte([spec], precision=G.MIXED)
    h.set_state(0, S.T, S.E, S.O)
    h.profile_begin(["pred_solve", "gmres"])
    h.step(1)
    prof = h.profile_end()
    assert prof.get("pred_solve", (0.0, 0))[1] == 1
    S1 = og.step(P, S)
    err = np.max(np.abs(h.T(0, allow=(5,)) - S1.T) / np.maximum(S1.T, 1e-300))
    print("mixed p = 2: %.2e" % err)
    assert err < 1e-5
    h.close()


def test_2d_fp64_vs_oracle_p1_5(G):
    mu, eta, w = s8_pairs_2d()
    n = 12
    rng = np.random.default_rng(5)
    sig = 0.5 + rng.random((n, n))
    P = og2.Problem2D(Nx=n, Ny=n, mu=mu, eta=eta, w=w, sig=sig, eps=1e-2, dt=0.4 / n, kind="t3", p=1.5, bx0=0.9)
    T0 = 0.2 + 0.5 * rng.random(n * n)
    h = G.Grte2D(n, n, sig, P.dt, P.eps, kind=G.SIGMA_POW, p=1.5, b_x0=0.9, mu=mu, eta=eta, w=w)
    h.set_state(T0)
    h.step(2, allow=(5,))
    S = og2.run(P, og2.equilibrium_state(P, T0), 2)
    err = np.max(np.abs(h.T(allow=(5,)) - S.T) / S.T)
    print("2D p = 1.5: %.2e" % err)
    assert err < 2e-11
    h.close()


def test_out_of_range_p_is_refused(G):
    _, spec = make(G, 64, 8, 1e-2, 3.5)
    with pytest.raises(G.GrteError) as e:
        G.Grte([spec])
    assert e.value.status == G.GRTE_EINVAL
