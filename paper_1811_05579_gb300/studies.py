"""Accuracy and stability studies of the scheme, run on the GPU path (FP64).

- convergence(): the l1 self-convergence of Sec. 6.2 (Eq. IC000 and Eq. error): sigma = 1,
  T(0, x) = max(1 - 40 (x - 1/2)^2, 0), I = a c T^4, zero inflow, dt = 0.1 dx, t = 0.1;
  error_rho and error_T between the solutions on dx and dx/2 (the fine one averaged to
  dx), for eps in {1, 1e-3, 1e-5} and dx = 1/25 .. 1/400.
- stability(): the largest C = dt/dx for which a run stays stable (the quantity of Tables
  stability1-2): Eq. IC000 data, zero inflow, run to t = 0.1, for sigma = 1 (Table
  stability1) and sigma = 1/T^3 (Table stability2).  The paper does not state its test of
  stability; here a run is stable when T stays finite, never exceeds the initial maximum
  (the limit equation's maximum principle) by more than 1e-6 relative, and ends with a
  single local maximum (the data are a single bump).
- marshak_dimensional(): the Marshak wave with units of Sec. 6.6 at the three time steps.
- long_run(): the slab configuration's 10^4 steps in FP64 and mixed precision side by side.

`python -m paper_1811_05579_gb300.studies` prints one JSON object with the first three
(`--long-run` adds the fourth)."""
import json
import math
import sys

import numpy as np

from . import grte as G
from . import workloads as wl


def _ic000(N):
    x = (np.arange(N) + 0.5) / N
    return np.maximum(1.0 - 40.0 * (x - 0.5) ** 2, 0.0)


def _spec(N, eps, dt, kind, n_dir=16):
    M = n_dir // 2
    return dict(nx=N, n_angle=M, sigma=np.ones(N), kind=kind, bc=G.BC_INFLOW, bL=np.zeros(M), bR=np.zeros(M),
                dt=dt, eps=eps)


def _run(N, eps, dt, kind, tmax, watch=False):
    """Advance Eq. IC000 data to tmax; returns (T, rho, max T seen, finite)."""
    h = G.Grte([_spec(N, eps, dt, kind)])
    T0 = _ic000(N)
    h.set_state(0, T0)
    steps = int(round(tmax / dt))
    tmax_seen, ok = float(T0.max()), True
    if watch:
        for _ in range(steps):
            h.step(1)
            T = h.T(0, allow=(5,))
            if not np.all(np.isfinite(T)):
                ok = False
                break
            tmax_seen = max(tmax_seen, float(T.max()))
    else:
        h.step(steps)
    T = h.T(0, allow=(5,))
    rho = h.rho(0, allow=(5,))
    h.close()
    return T, rho, tmax_seen, ok and bool(np.all(np.isfinite(T)))


def convergence(eps_list=(1.0, 1e-3, 1e-5), Ns=(25, 50, 100, 200, 400), tmax=0.1):
    out = {}
    for eps in eps_list:
        sols = {}
        for N in list(Ns) + [2 * Ns[-1]]:
            T, rho, _, _ = _run(N, eps, 0.1 / N, G.SIGMA_CONST, tmax)
            sols[N] = (T, rho)
        rows = []
        for N in Ns:
            eT = float(np.sum(np.abs(sols[N][0] - sols[2 * N][0].reshape(N, 2).mean(1))) / N)
            er = float(np.sum(np.abs(sols[N][1] - sols[2 * N][1].reshape(N, 2).mean(1))) / N)
            rows.append({"dx": 1.0 / N, "error_T": eT, "error_rho": er})
        for a, b in zip(rows[:-1], rows[1:]):
            b["rate_T"] = math.log2(a["error_T"] / b["error_T"])
            b["rate_rho"] = math.log2(a["error_rho"] / b["error_rho"])
        out["%g" % eps] = rows
    return out


def is_stable(N, eps, C, kind, tmax=0.1):
    T, _, seen, ok = _run(N, eps, C / N, kind, tmax, watch=True)
    if not ok:
        return False
    peaks = int(np.sum((T[1:-1] > T[:-2]) & (T[1:-1] >= T[2:]) & (T[1:-1] > 1e-8)))
    return seen <= 1.0 + 1e-6 and peaks <= 1


def stability(kind, eps_list=(1.0, 1e-3, 1e-5), Ns=(25, 50, 100, 200, 400),
              Cs=(0.1, 0.25, 0.5, 0.8, 1.0, 2.0, 4.0, 6.0, 8.0, 10.0, 16.0)):
    """Largest C of the list with a stable run (None: none stable), per (eps, dx)."""
    table = {}
    for eps in eps_list:
        row = {}
        for N in Ns:
            best = None
            for C in Cs:
                if is_stable(N, eps, C, kind):
                    best = C
                else:
                    break
            row["1/%d" % N] = best
        table["%g" % eps] = row
    return table


def marshak_dimensional(nx=50, t_end_ns=0.02):
    """The three time steps of Sec. 6.6 (1.6e-12, 8e-13, 4e-13 s): T at t_end and the
    position where T falls below 1/2 keV."""
    rows = []
    for dt_s in (1.6e-12, 8e-13, 4e-13):
        r = wl.marshak_dimensional(dt_s, nx=nx, t_end_ns=t_end_ns)
        h = G.Grte([dict(nx=r.nx, n_angle=r.n_dir // 2, sigma=r.sigma, kind=r.kind, bc=r.bc,
                         bL=np.full(r.n_dir // 2, r.bL), bR=np.full(r.n_dir // 2, r.bR), dt=r.dt, eps=r.eps,
                         a=r.a, c=r.c, Cv=r.Cv, x0=0.0, x1=r.length)])
        h.set_state(0, r.T0)
        h.step(r.steps)
        T = h.T(0, allow=(5,))
        h.close()
        x = (np.arange(r.nx) + 0.5) * r.length / r.nx
        rows.append({"dt_s": dt_s, "steps": r.steps, "T_max_keV": float(T.max()),
                     "half_keV_front_cm": float(x[int(np.argmax(T < 0.5))])})
    return rows


def long_run(steps=10000, chunk=1000):
    """The slab configuration's full run (six 8192-cell, 64-direction runs, dt = 0.5 dx,
    10^4 steps) in FP64 and in mixed precision side by side: per chunk of steps and per
    run, the largest T of each precision and their largest relative difference.  At this
    dt a run whose time step exceeds its stability limit (Tables stability1-3: the limit
    shrinks with dx) grows without bound, and rounding differences between the two
    precisions grow with it."""
    runs = wl.slab_1d_runs(steps=1)
    specs = [dict(nx=r.nx, n_angle=r.n_dir // 2, sigma=r.sigma, kind=r.kind, bc=r.bc,
                  bL=np.full(r.n_dir // 2, r.bL), bR=np.full(r.n_dir // 2, r.bR), dt=r.dt, eps=r.eps,
                  a=r.a, c=r.c, Cv=r.Cv) for r in runs]
    hd = G.Grte(specs)
    hm = G.Grte(specs, precision=G.MIXED)
    for i, r in enumerate(runs):
        hd.set_state(i, r.T0)
        hm.set_state(i, r.T0)
    rows = []
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        hd.step(n)
        hm.step(n)
        done += n
        row = {"step": done, "runs": []}
        for i, r in enumerate(runs):
            Td, Tm = hd.T(i, allow=(4, 5)), hm.T(i, allow=(4, 5))
            with np.errstate(all="ignore"):
                d = float(np.max(np.abs(Tm - Td) / np.maximum(np.abs(Td), 1e-300)))
            row["runs"].append({"sigma0": float(r.sigma[0]), "eps": r.eps, "T_max_fp64": float(np.max(Td)),
                                "T_max_mixed": float(np.max(Tm)), "t_rel_diff": d})
        rows.append(row)
    hd.close()
    hm.close()
    return rows


def main():
    res = {"convergence_sigma1": convergence(),
           "stability_sigma1": stability(G.SIGMA_CONST),
           "stability_sigma_T3": stability(G.SIGMA_T3),
           "marshak_dimensional": marshak_dimensional()}
    if "--long-run" in sys.argv:
        res["long_run_slab6"] = long_run()
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
