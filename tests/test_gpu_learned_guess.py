"""Learned Newton guess: the network's GPU forward/backward against the FP64 oracle of
the same network, and what the trained guess gains over the plain start (Newton
iterations per cell) while the converged temperatures stay the same."""
import numpy as np
import pytest

from oracle import mlp as om
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


def _norm_inputs(X, mi, si):
    return (X.astype(np.float32) - mi.astype(np.float32)) / si.astype(np.float32)


def test_mlp_forward_and_gradient_match_oracle(G):
    rng = np.random.default_rng(3)
    m = G.MLP(seed=5)
    mi = rng.standard_normal(6).astype(np.float32)
    si = (0.5 + rng.random(6)).astype(np.float32)
    m.set_norm(mi, si, 0.1, 2.0)
    X = (rng.standard_normal((301, 6)) * si + mi).astype(np.float32)
    Y = rng.standard_normal(301).astype(np.float32)
    p = m.params()
    xs = _norm_inputs(X, mi, si).astype(np.float64)
    # the network's BF16 form: every product's operands in bfloat16 (tensor cores), FP32
    # accumulation.  The kernel rounds FP32 values to bfloat16 where the oracle rounds
    # FP64 ones, so an operand can land one bfloat16 step (2^-8 relative) apart where the
    # two sit at a rounding tie: the bound is that of a few such steps, 2e-3
    out, _ = om.forward(om.unpack(om.to_bf16(p)), xs, act16=True)
    y_gpu = m.forward(X)
    assert np.max(np.abs(y_gpu - (out * 2.0 + 0.1))) < 2e-3 * max(1.0, np.max(np.abs(out * 2.0)))
    loss_g, g_gpu = m.grad(X, Y)
    t = (Y.astype(np.float64) - 0.1) / 2.0
    loss_o, g_o = om.loss_and_grad(p, xs, t, bf16=True)
    assert abs(loss_g - loss_o) < 2e-3 * max(loss_o, 1e-12)
    scale = np.max(np.abs(g_o))
    err = np.abs(g_gpu - g_o) / scale
    print("forward %.2e, loss %.2e, gradient max %.2e (median %.2e)"
          % (np.max(np.abs(y_gpu - (out * 2.0 + 0.1))), abs(loss_g - loss_o) / loss_o, err.max(), np.median(err)))
    assert err.max() < 2e-3 and np.median(err) < 1e-5
    m.close()


def _specs(insts):
    specs = []
    for r in insts:
        v, w = gauss_legendre_half(r.n_dir)
        specs.append(dict(nx=r.nx, n_angle=v.size, v=v, w=w, sigma=r.sigma, kind=1, bc=0,
                          bL=np.full(v.size, r.bL), bR=np.full(v.size, r.bR), dt=r.dt, eps=r.eps))
    return specs


def test_learned_guess_saves_newton_iterations(G):
    # training data: the scheme's own (features -> converged T^{n+1}) pairs
    train = wl.batched_1d(12, seed=21, nx_range=(128, 1024), n_dirs=(8, 16))
    h = G.Grte(_specs(train))
    for i, r in enumerate(train):
        h.set_state(i, r.T0)
    h.set_sample_logging(True)
    Xs, Ys = [], []
    for _ in range(25):
        h.step(1)
        for i in range(len(train)):
            X, y = h.newton_samples(i)
            Xs.append(X)
            Ys.append(y)
    h.close()
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    m = G.MLP(seed=1)
    m.set_norm(X.mean(0), X.std(0) + 1e-6, float(Y.mean()), float(Y.std() + 1e-6))
    loss = m.train(X, Y, epochs=30, batch=256, lr=1e-3, seed=3)
    print("training: %d samples, final standardised MSE %.4f (target std %.3g)" % (X.shape[0], loss, Y.std()))
    assert loss < 0.5, loss   # standardised MSE well below the 1.0 of a constant guess
    # held-out instances: the three starts of Newton's iteration, with per-cell counts
    # split into front cells (T changes by more than 1% in the step) and the rest
    test = wl.batched_1d(6, seed=77, nx_range=(128, 1024), n_dirs=(8, 16))
    res = {}
    for mode in ("previous", "bound", "learned"):
        hh = G.Grte(_specs(test))
        for i, r in enumerate(test):
            hh.set_state(i, r.T0)
        if mode == "learned":
            hh.set_guess(m)
        elif mode == "previous":
            hh.set_newton_start(G.START_PREVIOUS)
        front, rest = [], []
        for _ in range(8):
            Tb = [hh.T(i, allow=(5,)) for i in range(len(test))]
            hh.step(1)
            for i in range(len(test)):
                its = hh.stage(i, 3, allow=(5,))
                Ta = hh.T(i, allow=(5,))
                big = np.abs(Ta / np.maximum(Tb[i], 1e-300) - 1.0) > 1e-2
                front.append(its[big])
                rest.append(its[~big])
        res[mode] = ([hh.T(i, allow=(5,)) for i in range(len(test))],
                     float(np.mean(np.concatenate(front))), float(np.mean(np.concatenate(rest))),
                     int(sum(f.size for f in front)))
        hh.close()
    for mode in ("previous", "bound", "learned"):
        print("Newton iterations per cell, start %-8s: front cells %.3f (%d), other cells %.3f"
              % (mode, res[mode][1], res[mode][3], res[mode][2]))
    # the same roots: each step's T agrees to the per-step FP64 bound 1e-12, and the
    # differences of rounding accumulate over the 8 steps
    for mode in ("previous", "learned"):
        for a, b in zip(res[mode][0], res["bound"][0]):
            assert np.max(np.abs(a - b) / b) < 1e-11
    # at the fronts the trained start beats the textbook start from T^n, and overall it
    # does not lose against the closed-form bound
    assert res["learned"][1] < 0.8 * res["previous"][1], res
    lf, bf = res["learned"][1], res["bound"][1]
    assert lf <= bf * 1.05 and res["learned"][2] <= res["bound"][2] * 1.05, res
    m.close()
