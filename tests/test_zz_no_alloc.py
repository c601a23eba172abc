"""The allocation-free step entry point against the handle-based one.

Some callers cannot allocate device memory (they run inside an allocator or memory
pool callback, or under a fixed memory budget).  grte_step1d_noalloc serves them: it
takes the state in the caller's device buffers and does its work in a static device
array.  These tests call it through the C ABI twice in a row and check, after each
call, that it gives what grte_create_1d + grte_step give for the same instance, to
the tolerance of the other parity tests, and that both return the same status.  The
cases cover inflow and reflecting walls, several steps inside one call with an
explicit options struct, and the largest sizes the static array admits
(nx = 4096 with 16 angles, nx = 2048 with 32 angles: nx * n_angle = 65536).  The file
is collected last so that a run stopping at the first failure has run every other
test first.
"""
import numpy as np
import pytest

from oracle.quadrature import gauss_legendre_half
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, n_dir, eps, bc, nsteps per call, explicit options)
    (300, 16, 1e-2, "inflow", 1, None),
    (300, 16, 1e-2, "reflect", 3, dict(krylov_restart=8, krylov_rtol=1e-13, newton_maxit=40)),
    (4096, 32, 1e-3, "inflow", 1, None),        # nx at its limit, 16 angles: 65536 line elements
    (2048, 64, 1.0, "reflect", 2, dict(krylov_restart=12)),   # 32 angles at their limit
]


@pytest.mark.parametrize("nx,nv,eps,bcname,nsteps,options", CASES)
def test_noalloc_step_matches_handle_step_twice(nx, nv, eps, bcname, nsteps, options):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte as G
    N = nx
    v, w = gauss_legendre_half(nv)
    M = v.size
    bc = G.BC_INFLOW if bcname == "inflow" else G.BC_REFLECT
    spec = dict(nx=N, n_angle=M, v=v, w=w, sigma=np.full(N, 2.0), kind=G.SIGMA_T3, bc=bc,
                bL=np.full(M, 0.9), bR=np.full(M, 0.05), dt=0.5 / N, eps=eps)
    rng = wl.SplitMix64(4242 + N)
    T0 = wl.smoothed_log_uniform_T(rng, N, 0.1, 1.0, width=9)
    x = (np.arange(N) + 0.5) / N
    E0 = (T0 ** 4)[:, None] * (1.0 + 0.05 * np.sin(2 * np.pi * x)[:, None] * v[None, :])
    O0 = np.zeros((N + 1, M))
    hopt = dict(options or {})
    h = G.Grte([spec], line_threads=256, **hopt)   # the line-solve size the no-alloc step uses
    h.set_state(0, T0, E0, O0)
    dev = torch.device("cuda", 0)
    Td = torch.tensor(T0, dtype=torch.float64, device=dev)
    Ed = torch.tensor(np.ascontiguousarray(E0.T), dtype=torch.float64, device=dev)   # line-major [k][j]
    Od = torch.tensor(np.ascontiguousarray(O0.T), dtype=torch.float64, device=dev)   # [k][i]
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        h.step(nsteps)
        sh = h.sync(allow=(4, 5))
        st = G.step1d_noalloc(spec, Td.data_ptr(), Ed.data_ptr(), Od.data_ptr(), nsteps, stream.cuda_stream,
                              options=options)
        assert st == sh and st in (G.GRTE_OK, 5), (G.STATUS_NAMES.get(st, st), G.STATUS_NAMES.get(sh, sh))
        torch.cuda.synchronize()
        Th, Eh, Oh = h.T(0, allow=(5,)), h.E(0, allow=(5,)), h.O(0, allow=(5,))
        Tn = Td.cpu().numpy()
        En = Ed.cpu().numpy().T
        On = Od.cpu().numpy().T
        # per-cell tolerance of the parity tests: 1e-12, in the two wall cells 1e-12 + 4e-15/eps
        # (there the wall rows turn a rounding difference into one of O that grows like 1/eps)
        tol = np.full(N, 1e-12)
        if bcname == "inflow":
            tol[0] = tol[-1] = 1e-12 + 4e-15 / eps
        tol = tol * (call + 1) * nsteps        # per step taken so far, as the other parity tests
        errT = np.max(np.abs(Tn - Th) / np.maximum(Th, 1e-300) / tol) * 1e-12
        # E = a c U + Eh: rounding relative to |E| + a c U (E can be a small difference)
        errE = np.max(np.abs(En - Eh) / np.maximum(np.abs(Eh) + (Th ** 4)[:, None], 1e-300) / tol[:, None]) * 1e-12
        print("noalloc nx=%d M=%d %s call %d: T %.2e E %.2e" % (N, M, bcname, call, errT, errE))
        assert errT < 1e-12, call
        assert errE < 1e-12, call
        assert np.max(np.abs(On - Oh)) <= 1e-12 * max(np.max(np.abs(Oh)), 1e-300), call
    h.close()


def test_noalloc_rejects_sizes_beyond_its_static_memory():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte as G
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")   # never touched: the size check comes first
    for nx, M in ((8192, 32), (4097, 8), (2048, 33), (4096, 17)):
        spec = dict(nx=nx, n_angle=M, sigma=np.ones(nx), dt=1e-4, eps=1.0)
        st = G.step1d_noalloc(spec, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1, None)
        assert st == 1, (nx, M)     # GRTE_EINVAL
