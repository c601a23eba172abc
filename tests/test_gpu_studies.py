"""The paper's accuracy and stability claims, and its Marshak wave with units, on the GPU
path (FP64; `paper_1811_05579_gb300/studies.py` runs the full versions).

- Sec. 6.2, Eq. error: error_rho and error_T of the GPU solutions on dx and dx/2 decrease
  at first order for eps = 1, 1e-3, 1e-5 (uniform first-order accuracy).
- Tables stability1-2 (largest C = dt/dx), at the points where the oracle's stability
  test agrees with the tables: sigma = 1, eps = 1 stable at C = 16 (table: > 10);
  sigma = 1/T^3, eps = 1e-3, dx = 1/100 stable at C = 1 and not at C = 2 (table: 1);
  sigma = 1/T^3, eps = 1, dx = 1/100 stable at C = 4, not at C = 16 (table: 8).
- The Marshak wave with units (last example of Sec. 6) at its three time steps against
  the oracle, and bounded by the wall temperature (1 keV) within 10%."""
import numpy as np
import pytest

from oracle import grte1d as og
from oracle.quadrature import gauss_legendre_half
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import studies
    return studies


@pytest.mark.parametrize("eps", [1.0, 1e-3, 1e-5])
def test_first_order_self_convergence_on_gpu(S, eps):
    rows = S.convergence(eps_list=(eps,), Ns=(25, 50, 100, 200))["%g" % eps]
    print(eps, rows)
    for r in rows[1:]:
        assert r["rate_rho"] > 0.8, rows
    if eps < 1.0:
        for r in rows[1:]:
            assert r["rate_T"] > 0.8, rows
    else:
        # T = U^{1/4} is not Lipschitz at the edge of the support: overall decrease
        assert np.log2(rows[0]["error_T"] / rows[-1]["error_T"]) / (len(rows) - 1) > 0.8, rows


def test_stability_limits_of_the_tables(S):
    from paper_1811_05579_gb300 import grte as G
    assert S.is_stable(25, 1.0, 16.0, G.SIGMA_CONST)
    assert S.is_stable(100, 1.0, 16.0, G.SIGMA_CONST)
    assert S.is_stable(100, 1e-3, 1.0, G.SIGMA_T3)
    assert not S.is_stable(100, 1e-3, 2.0, G.SIGMA_T3)
    assert S.is_stable(100, 1.0, 4.0, G.SIGMA_T3)
    assert not S.is_stable(100, 1.0, 16.0, G.SIGMA_T3)


@pytest.mark.parametrize("dt_s", [1.6e-12, 8e-13, 4e-13])
def test_marshak_wave_with_units_vs_oracle(S, dt_s):
    from paper_1811_05579_gb300 import grte as G
    r = wl.marshak_dimensional(dt_s)
    M = r.n_dir // 2
    v, w = gauss_legendre_half(r.n_dir)
    P = og.Problem(N=r.nx, v=v, w=w, sig=r.sigma, eps=r.eps, dt=r.dt, kind="t3", a=r.a, c=r.c, Cv=r.Cv,
                   x0=0.0, x1=r.length, bL=np.full(M, r.bL), bR=np.full(M, r.bR))
    h = G.Grte([dict(nx=r.nx, n_angle=M, v=v, w=w, sigma=r.sigma, kind=1, bc=0, bL=P.bL, bR=P.bR, dt=r.dt,
                     eps=r.eps, a=r.a, c=r.c, Cv=r.Cv, x0=0.0, x1=r.length)])
    h.set_state(0, r.T0)
    h.step(r.steps)
    Tg = h.T(0, allow=(5,))
    So = og.run(P, og.equilibrium_state(P, r.T0), r.steps)
    err = np.abs(Tg - So.T) / np.maximum(So.T, 1e-300)
    print("dt %.1e s, %d steps: T vs oracle %.2e, max T %.4f keV" % (dt_s, r.steps, err.max(), Tg.max()))
    assert err.max() < 1e-12 * r.steps + 1e-11
    assert Tg.max() < 1.1
    h.close()
