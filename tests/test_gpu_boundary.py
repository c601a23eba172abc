"""The C ABI's checkpoint, device hand-off and status paths, driven from the host.

- grte_get_state / grte_restore_state: a restored handle continues bit for bit (FP64
  line kernels, mixed one-kernel solve, mixed line kernels); blobs of another precision,
  other sizes or truncated are refused (EINVAL).
- grte_get_T_device: T copied into a caller's CUDA buffer on the caller's stream.
- grte_create: one call for 1D and 2D problems, the same handles as the per-dimension calls.
- Status paths, each caused on the host: NaN in the state (injected through a blob,
  since grte_set_state refuses non-finite T with EINVAL) -> ENAN; newton_maxit = 1 and
  krylov_maxcycles = 1 -> ENONCONV, reported by every grte_get_* call until grte_sync
  has returned it; a wrong len -> EINVAL; an injected allocation failure -> ENOMEM.
No test here faults, traps or hangs the device: the failures are made by the inputs."""
import struct

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


def spec(N, nv=16, eps=1e-2, bL=1.0):
    v, w = gauss_legendre_half(nv)
    return dict(nx=N, n_angle=v.size, v=v, w=w, sigma=np.full(N, 2.0), kind=1, bc=0,
                bL=np.full(v.size, bL), bR=np.zeros(v.size), dt=0.5 / N, eps=eps)


def T0(N, seed=3):
    return wl.smoothed_log_uniform_T(wl.SplitMix64(seed + N), N, 0.05, 0.5, width=9)


@pytest.mark.parametrize("prec,solver", [("fp64", "auto"), ("mixed", "auto"), ("mixed", "lines")])
def test_restore_continues_bit_for_bit(G, prec, solver):
    specs = [spec(700), spec(96, nv=8, eps=1e-4)]
    kw = dict(precision=G.MIXED if prec == "mixed" else G.FP64,
              solver1d=G.SOLVER_LINES if solver == "lines" else G.SOLVER_AUTO, energy_every=1)
    a = G.Grte(specs, **kw)
    for i, s in enumerate(specs):
        a.set_state(i, T0(s["nx"], i))
    a.step(3)
    blob = a.get_state(allow=(5,))
    a.step(2)
    b = G.Grte(specs, **kw)
    b.restore_state(blob)
    b.step(2)
    for i in range(len(specs)):
        assert np.array_equal(a.T(i, allow=(5,)), b.T(i, allow=(5,)))
        assert np.array_equal(a.E(i, allow=(5,)), b.E(i, allow=(5,)))
        assert np.array_equal(a.O(i, allow=(5,)), b.O(i, allow=(5,)))
        assert np.array_equal(a.energy(i), b.energy(i))
    assert a.stats(allow=(5,))["steps"] == b.stats(allow=(5,))["steps"] == 5
    # refused: another precision, other sizes, a truncated blob
    c = G.Grte(specs, precision=G.FP64 if prec == "mixed" else G.MIXED)
    with pytest.raises(G.GrteError) as e:
        c.restore_state(blob)
    assert e.value.status == G.GRTE_EINVAL
    d = G.Grte([spec(700), spec(97, nv=8)], **kw)
    with pytest.raises(G.GrteError) as e:
        d.restore_state(blob)
    assert e.value.status == G.GRTE_EINVAL
    with pytest.raises(G.GrteError) as e:
        b.restore_state(blob[:-8])
    assert e.value.status == G.GRTE_EINVAL
    for h in (a, b, c, d):
        h.close()


def test_T_device_on_the_callers_stream(G):
    import torch
    N = 300
    h = G.Grte([spec(N)])
    h.set_state(0, T0(N))
    h.step(2)
    s = torch.cuda.Stream()
    out = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    h.T_device(0, out.data_ptr(), N, s.cuda_stream)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), h.T(0, allow=(5,)))
    h.sync(allow=(5,))
    with pytest.raises(G.GrteError) as e:
        h.T_device(0, out.data_ptr(), N - 1)
    assert e.value.status == G.GRTE_EINVAL
    h.close()


def _t_offset(blob, inst_sizes):
    """Byte offset of T of instance 0 in a state blob (header, per-instance sizes,
    energy sums)."""
    head = 8 + 4 * 4 + 8
    n_inst = struct.unpack_from("<I", blob, 8 + 12)[0]
    assert n_inst == len(inst_sizes)
    return head + 16 * n_inst + 24 * n_inst


def test_nan_state_reports_enan_until_synced(G):
    N = 200
    h = G.Grte([spec(N)])
    with pytest.raises(G.GrteError) as e:
        T = T0(N)
        T[7] = np.nan
        h.set_state(0, T)
    assert e.value.status == G.GRTE_EINVAL            # the setter checks its input
    h.set_state(0, T0(N))
    blob = bytearray(h.get_state())
    off = _t_offset(blob, [N]) + 8 * 7
    struct.pack_into("<d", blob, off, float("nan"))
    h.restore_state(bytes(blob))
    h.step(1)
    with pytest.raises(G.GrteError) as e:
        h.T(0)                                        # reported by the getters ...
    assert e.value.status == G.GRTE_ENAN
    with pytest.raises(G.GrteError) as e:
        h.sync()                                      # ... and by grte_sync, which clears it
    assert e.value.status == G.GRTE_ENAN
    assert h.sync() == G.GRTE_OK
    h.close()


@pytest.mark.parametrize("what", ["newton", "krylov"])
def test_iteration_limits_report_enonconv(G, what):
    N = 400
    kw = dict(newton_maxit=1) if what == "newton" else dict(krylov_maxcycles=1, krylov_rtol=1e-16)
    h = G.Grte([spec(N, eps=1e-3)], **kw)
    h.set_state(0, T0(N))
    h.step(2)
    with pytest.raises(G.GrteError) as e:
        h.E(0)
    assert e.value.status == G.GRTE_ENONCONV
    with pytest.raises(G.GrteError) as e:
        h.T(0)                                        # sticky until grte_sync
    assert e.value.status == G.GRTE_ENONCONV
    with pytest.raises(G.GrteError) as e:
        h.sync()
    assert e.value.status == G.GRTE_ENONCONV
    assert h.sync() == G.GRTE_OK
    h.close()


def test_wrong_lengths_are_einval(G):
    import ctypes
    N = 128
    h = G.Grte([spec(N)])
    h.set_state(0, T0(N))
    L = G.lib()
    buf = np.zeros(4 * N * 16)
    for fn, n in ((L.grte_get_T, N + 1), (L.grte_get_rho, N - 1), (L.grte_get_E, N * 8 + 1),
                  (L.grte_get_O, N * 8)):
        assert fn(h.h, 0, G._ptr(buf), n) == G.GRTE_EINVAL
    assert L.grte_get_T(h.h, 1, G._ptr(buf), N) == G.GRTE_EINVAL          # no instance 1
    n = ctypes.c_size_t(10)
    assert L.grte_get_state(h.h, G._ptr(buf), ctypes.byref(n)) == G.GRTE_EINVAL   # too small
    h.close()


def test_injected_allocation_failure_is_enomem(G):
    for after in (0, 5, 40):
        G.lib().grte_test_fail_alloc_after(after)
        try:
            with pytest.raises(G.GrteError) as e:
                G.Grte([spec(256)])
            assert e.value.status == G.GRTE_ENOMEM
        finally:
            G.lib().grte_test_fail_alloc_after(-1)
    h = G.Grte([spec(256)])                           # allocations work again
    h.set_state(0, T0(256))
    h.step(1)
    assert h.sync(allow=(5,)) in (G.GRTE_OK, 5)
    h.close()


def test_one_create_call_for_both_dimensions(G):
    """grte_create builds the same 1D and 2D handles as grte_create_1d and grte2d_create
    (steps bit-identical); an unknown dimension or mismatched edge kinds are EINVAL."""
    N = 256
    v, w = gauss_legendre_half(16)
    p1 = G.Problem(1, N, 0.5 / N, 1e-2, 2.0, n_dir=16, mu=v, w=w, b_iso=(1.0, 0.0, 0.0, 0.0))
    ref = G.Grte([spec(N)])
    T = T0(N)
    p1.set_initial(T)
    ref.set_state(0, T)
    p1.step(3)
    ref.step(3)
    assert np.array_equal(p1.T(allow=(5,)), ref.T(0, allow=(5,)))
    p1.close()
    ref.close()
    n = 24
    sig = 1.0 + 9.0 * ((np.arange(n)[:, None] // 8 + np.arange(n)[None, :] // 8) % 2)
    T2 = 1e-2 * (1.0 + 0.5 * wl.SplitMix64(5).uniform(n * n))
    p2 = G.Problem(2, n, 0.5 / n, 1e-3, sig, ny=n, b_iso=(1.0, 0.0, 0.0, 0.0))
    r2 = G.Grte2D(n, n, sig, 0.5 / n, 1e-3, b_x0=1.0, krylov_restart=10)
    p2.set_initial(T2)
    r2.set_state(T2)
    p2.step(2)
    r2.step(2, allow=(5,))
    assert np.array_equal(p2.T(allow=(5,)), r2.T(allow=(5,)))
    p2.close()
    r2.close()
    with pytest.raises(G.GrteError) as e:
        G.Problem(3, N, 0.5 / N, 1e-2, 2.0)
    assert e.value.status == G.GRTE_EINVAL
    with pytest.raises(G.GrteError) as e:
        G.Problem(1, N, 0.5 / N, 1e-2, 2.0, bc_kind=(G.BC_INFLOW, G.BC_REFLECT, 0, 0))
    assert e.value.status == G.GRTE_EINVAL
