"""The three-stage diffusion solver of Sec. 2 on the GPU (grte_diff_*) against the
oracle's (Eq. dis-diff; sigma_0/T^3: the fully discrete form after Eq. marshak-diff2):
uneven batches of both opacity forms, steps from compactly supported and smooth data,
U* and T per cell to 1e-12 relative per step; the bound R <= 0 status; bad lengths."""
import numpy as np
import pytest

from oracle import diffusion1d as dif
from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte
    return grte


def test_three_stage_solver_vs_oracle(G):
    rng = wl.SplitMix64(812)
    insts = []
    for N, kind, dt in ((100, "const", 0.005 / 100), (257, "t3", 0.1 / 257), (1000, "const", 0.5 / 1000),
                        (3000, "t3", 0.05 / 3000)):
        x = (np.arange(N) + 0.5) / N
        T0 = np.maximum(np.sin(2 * np.pi * (x - 0.25)), 0.0) ** 0.25 if kind == "const" else \
            np.maximum(1.0 - 40.0 * (x - 0.5) ** 2, 0.0) + 1e-3
        sig = 0.2 + 2.0 * rng.uniform(N)
        insts.append(dict(nx=N, sigma=sig, kind=G.SIGMA_CONST if kind == "const" else G.SIGMA_T3, dt=dt,
                          a=1.0, c=1.0, Cv=1.0, T0=T0, okind=kind))
    h = G.Diffusion(insts)
    for i, p in enumerate(insts):
        h.set_T(i, p["T0"])
    steps = 5
    h.step(steps)
    for i, p in enumerate(insts):
        T = p["T0"].copy()
        for _ in range(steps):
            T, Us = dif.three_stage_step(T, p["sigma"], 1.0 / p["nx"], p["dt"], kind=p["okind"])
        Tg = h.T(i, allow=(5,))
        Ug = h.Ustar(i, allow=(5,))
        scale = np.max(np.abs(T))
        eT = np.max(np.abs(Tg - T)) / scale
        eU = np.max(np.abs(Ug - Us)) / np.max(np.abs(Us))
        print("inst %d N=%d %s: T %.2e U* %.2e" % (i, p["nx"], p["okind"], eT, eU))
        assert eT < 1e-12 * steps and eU < 1e-12 * steps
    h.close()


def test_lengths_and_values_are_checked(G):
    h = G.Diffusion([dict(nx=64, sigma=1.0, dt=1e-3)])
    with pytest.raises(G.GrteError) as e:
        h.set_T(0, np.ones(63))
    assert e.value.status == G.GRTE_EINVAL
    with pytest.raises(G.GrteError) as e:
        h.set_T(0, -np.ones(64))
    assert e.value.status == G.GRTE_EINVAL
    with pytest.raises(G.GrteError) as e:
        G.Diffusion([dict(nx=64, sigma=0.0, dt=1e-3)])
    assert e.value.status == G.GRTE_EINVAL
    h.close()
