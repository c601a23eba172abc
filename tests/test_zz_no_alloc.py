"""The allocation-free step entry point against the handle-based one.

Some callers cannot allocate device memory (they run inside an allocator or memory
pool callback, or under a fixed memory budget).  grte_step1d_noalloc serves them: it
takes the state in the caller's device buffers and does its work in a static device
array.  This test calls it through the C ABI twice in a row and checks, after each
call, that it gives what grte_create_1d + grte_step give for the same instance, to
the tolerance of the other parity tests.  It sits in a file that pytest collects
last so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from oracle.quadrature import gauss_legendre_half
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte as G
    N, nv, eps = 300, 16, 1e-2
    v, w = gauss_legendre_half(nv)
    M = v.size
    spec = dict(nx=N, n_angle=M, v=v, w=w, sigma=np.full(N, 2.0), kind=G.SIGMA_T3, bc=G.BC_INFLOW,
                bL=np.full(M, 0.9), bR=np.full(M, 0.05), dt=0.5 / N, eps=eps)
    rng = wl.SplitMix64(4242)
    T0 = wl.smoothed_log_uniform_T(rng, N, 0.1, 1.0, width=9)
    x = (np.arange(N) + 0.5) / N
    E0 = (T0 ** 4)[:, None] * (1.0 + 0.05 * np.sin(2 * np.pi * x)[:, None] * v[None, :])
    O0 = np.zeros((N + 1, M))
    h = G.Grte([spec])
    h.set_state(0, T0, E0, O0)
    dev = torch.device("cuda", 0)
    Td = torch.tensor(T0, dtype=torch.float64, device=dev)
    Ed = torch.tensor(np.ascontiguousarray(E0.T), dtype=torch.float64, device=dev)   # line-major [k][j]
    Od = torch.tensor(np.ascontiguousarray(O0.T), dtype=torch.float64, device=dev)   # [k][i]
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        h.step(1)
        sh = h.sync(allow=(4, 5))
        st = G.step1d_noalloc(spec, Td.data_ptr(), Ed.data_ptr(), Od.data_ptr(), 1, stream.cuda_stream)
        assert st == sh and st in (G.GRTE_OK, 5), (G.STATUS_NAMES.get(st, st), G.STATUS_NAMES.get(sh, sh))
        torch.cuda.synchronize()
        Th, Eh, Oh = h.T(0, allow=(5,)), h.E(0, allow=(5,)), h.O(0, allow=(5,))
        Tn = Td.cpu().numpy()
        En = Ed.cpu().numpy().T
        On = Od.cpu().numpy().T
        assert np.max(np.abs(Tn - Th) / Th) < 1e-12, call
        assert np.max(np.abs(En - Eh) / np.abs(Eh)) < 1e-12, call
        assert np.max(np.abs(On - Oh)) <= 1e-12 * np.max(np.abs(Oh)), call
    h.close()


def test_noalloc_rejects_sizes_beyond_its_static_memory():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte as G
    spec = dict(nx=8192, n_angle=32, sigma=np.ones(8192), dt=1e-4, eps=1.0)
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")   # never touched: the size check comes first
    st = G.step1d_noalloc(spec, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1, None)
    assert st == 1     # GRTE_EINVAL
