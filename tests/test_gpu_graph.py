"""The captured step (one CUDA graph launch per step, Krylov loop under device-side
conditional nodes) against the eager step (host loop): the same kernels run on the
same data in the same order, so the states agree bit for bit."""
import numpy as np
import pytest

from oracle.quadrature import gauss_legendre_half
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte
    return grte


def _specs(insts):
    out = []
    for r in insts:
        v, w = gauss_legendre_half(r.n_dir)
        out.append(dict(nx=r.nx, n_angle=v.size, v=v, w=w, sigma=r.sigma, kind=r.kind, bc=r.bc,
                        bL=np.full(v.size, r.bL), bR=np.full(v.size, r.bR), dt=r.dt, eps=r.eps))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_step_equals_eager_step(G, precision):
    insts = wl.batched_1d(5, seed=31, nx_range=(64, 700), n_dirs=(8, 16)) + [wl.marshak_1d()]
    specs = _specs(insts)
    prec = G.FP64 if precision == "fp64" else G.MIXED
    res = {}
    for use_graph in (False, True):
        # one line-thread count for both (the autotuner times the candidates per handle)
        h = G.Grte(specs, precision=prec, use_graph=use_graph, line_threads=256)
        for i, r in enumerate(insts):
            h.set_state(i, r.T0)
        its = []
        for _ in range(4):
            h.step(2)
            st = h.stats(allow=(5,))
            its.append((st["krylov_iters"], st["krylov_cycles"]))
            assert h.last_launches() > 0
        res[use_graph] = ([h.T(i, allow=(5,)) for i in range(len(insts))],
                          [h.E(i, allow=(5,)) for i in range(len(insts))],
                          [h.O(i, allow=(5,)) for i in range(len(insts))], its)
        h.close()
    for q in range(3):
        for a, b in zip(res[False][q], res[True][q]):
            assert np.array_equal(a, b)
    assert res[False][3] == res[True][3]


def test_graph_rebuilt_after_newton_start_change(G):
    insts = [wl.marshak_1d()]
    specs = _specs(insts)
    out = []
    for use_graph in (False, True):
        h = G.Grte(specs, use_graph=use_graph, line_threads=256)
        h.set_state(0, insts[0].T0)
        h.step(3)
        h.set_newton_start(G.START_PREVIOUS)   # changes a value the captured kernels take
        h.step(3)
        out.append((h.T(0, allow=(5,)), h.stage(0, 3, allow=(5,))))
        h.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
