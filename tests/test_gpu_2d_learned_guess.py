"""Learned Newton start on the 2D path: the network is trained on the (features ->
log10 T^{n+1}/T^n) pairs that 2D checkerboard runs log on the GPU, then started on a
held-out random-smooth (log-normal sigma_0) problem.  Newton iterations per cell are
compared with the previous-T and closed-form-bound starts; the temperatures agree."""
import numpy as np
import pytest

from paper_1811_05579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_05579_gb300 import grte
    return grte


def _handle(G, sig, n, eps, T0):
    h = G.Grte2D(n, n, sig, 0.5 / n, eps, kind=G.SIGMA_T3, b_x0=1.0)
    h.set_state(T0)
    return h


def test_2d_sample_logging_features(G):
    n = 16
    sig = wl.checkerboard_sigma_2d(n, blocks=4)
    T0 = np.full(n * n, 1e-2)
    h = _handle(G, sig, n, 1e-3, T0)
    h.set_sample_logging(True)
    h.step(1, allow=(5,))
    X, y = h.newton_samples()
    T1 = h.T(allow=(5,))
    rho = h.stage(2, allow=(5,))
    ok = (T1 > 0) & (rho > 0)
    assert np.allclose(X[:, 0], np.log10(T0), rtol=0, atol=1e-6)
    assert np.allclose(X[ok, 1], np.log10(rho[ok]), rtol=0, atol=1e-5)
    assert np.allclose(X[:, 2], np.log10(sig.ravel() / T0 ** 3), rtol=0, atol=1e-5)
    assert np.allclose(X[:, 3:], np.log10([1e-3, 0.5 / n, 1.0])[None, :], rtol=0, atol=1e-6)
    assert np.allclose(y[ok], np.log10(T1[ok] / T0[ok]), rtol=0, atol=1e-6)
    h.close()


def test_2d_learned_start_saves_newton_iterations(G):
    # training: the scheme's own pairs from runs of two families on 24^2..56^2 grids (so
    # that the dt feature varies): checkerboards (8 x 8 board) whose two sigma_0 values
    # are drawn per run, log-uniform in [10^-0.5, 1] and [10, 100], and log-normal sigma_0
    # fields of other seeds; eps 1e-3 and 1e-4; the initial temperature 1e-2 times a
    # seeded factor in [1, 1.5)
    runs = []
    for r, n in enumerate((24, 32, 40, 56)):
        u = wl.SplitMix64(wl.BASE_SEED + 100 + r).uniform(2)
        runs.append((n, wl.checkerboard_sigma_2d(n, lo=10 ** (-0.5 + 0.5 * u[0]), hi=10 ** (1.0 + u[1])),
                     1e-3 if r % 2 == 0 else 1e-4, 41 + r))
    for r, n in enumerate((32, 40)):
        runs.append((n, wl.lognormal_sigma_2d(n, seed=wl.BASE_SEED + 11 + r, sd_cells=3.0), 1e-4, 51 + r))
    Xs, Ys = [], []
    for n, sig, eps, seed in runs:
        T0 = 1e-2 * (1.0 + 0.5 * wl.SplitMix64(seed).uniform(n * n))
        h = _handle(G, sig, n, eps, T0)
        h.set_sample_logging(True)
        for _ in range(25):
            h.step(1, allow=(5,))
            X, y = h.newton_samples()
            keep = np.all(np.isfinite(X), axis=1) & (X[:, 0] > -30) & (np.abs(X[:, 2]) < 30)
            Xs.append(X[keep])
            Ys.append(y[keep])
        h.close()
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    m = G.MLP(seed=1)
    # a floor on the feature scales: eps and Cv take few values in the training runs, and a
    # near-zero scale would blow up any value not seen there
    m.set_norm(X.mean(0), np.maximum(X.std(0), 0.1), float(Y.mean()), float(Y.std() + 1e-6))
    loss = m.train(X, Y, epochs=30, batch=256, lr=1e-3, seed=3)
    print("training: %d samples, final standardised MSE %.4f (target std %.3g)" % (X.shape[0], loss, Y.std()))
    assert loss < 0.5, loss
    # held out: a log-normal sigma_0 field of another seed (Gaussian-smoothed, sd 4 cells), eps 1e-4
    nt = 48
    sig = wl.lognormal_sigma_2d(nt, seed=wl.BASE_SEED + 7, sd_cells=4.0)
    T0 = np.full(nt * nt, 1e-2)
    res = {}
    for mode in ("previous", "bound", "learned"):
        hh = _handle(G, sig, nt, 1e-4, T0)
        if mode == "learned":
            hh.set_guess(m)
            hh.set_sample_logging(True)
        elif mode == "previous":
            hh.set_newton_start(G.START_PREVIOUS)
        front, rest, perr = [], [], []
        for _ in range(8):
            Tb = hh.T(allow=(5,))
            hh.step(1, allow=(5,))
            its = hh.stage(3, allow=(5,))
            Ta = hh.T(allow=(5,))
            big = np.abs(Ta / np.maximum(Tb, 1e-300) - 1.0) > 1e-2
            front.append(its[big])
            rest.append(its[~big])
            if mode == "learned":
                X, y = hh.newton_samples()
                perr.append((m.forward(X) - y)[big])
        if perr:
            e = np.concatenate(perr)
            print("held-out front cells: network error in log10 T, RMS %.3g, 90th percentile %.3g"
                  % (np.sqrt(np.mean(e ** 2)), np.quantile(np.abs(e), 0.9)))
        res[mode] = (hh.T(allow=(5,)), float(np.mean(np.concatenate(front))),
                     float(np.mean(np.concatenate(rest))), int(sum(f.size for f in front)))
        hh.close()
    for mode in ("previous", "bound", "learned"):
        print("Newton iterations per cell, start %-8s: front cells %.3f (%d), other cells %.3f"
              % (mode, res[mode][1], res[mode][3], res[mode][2]))
    # the same roots: every step's Krylov solve stops at 1e-13 of its scaled residual, so
    # two runs whose Newton roots differ in the last bits agree to the 2D parity bound
    # (1e-11 per step), accumulated over the 8 steps
    for mode in ("previous", "learned"):
        d = float(np.max(np.abs(res[mode][0] - res["bound"][0]) / np.maximum(res["bound"][0], 1e-300)))
        print("max relative T difference, %s vs bound: %.3e" % (mode, d))
        assert d < 1e-10, (mode, d)
    assert res["learned"][1] < 0.8 * res["previous"][1], res
    assert res["learned"][1] <= 1.05 * res["bound"][1] and res["learned"][2] <= 1.05 * res["bound"][2], res
    m.close()
