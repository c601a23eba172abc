"""Throughput of the 1D AP step (cell-angle updates/s) on GB300.

Workload (default): the 1D slab runs - 8192 cells, Gauss-Legendre 64 directions
(32 +-v pairs), sigma = sigma0/T^3 with sigma0 in {1, 10} x eps in {1, 1e-2, 1e-4}
(six independent runs advanced together in one handle), T_in log-uniform in
[1e-3, 1e-2] then smoothed, left inflow a c 1^4, right vacuum, dt = 0.5 dx.  A
step advances all six runs by one time step of Algorithm 2.  Inputs are seeded
synthetic data; the state is resident in HBM before timing starts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank runs its own six runs (weak
scaling); the timed region is bracketed by barriers and the max over ranks is used.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "cell-angle updates/s"
UNIT = "cell-angle updates/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_PEAK_GFLOPS = 1250.0           # nominal GB300 FP64 (the profiling recipe's figure)

# Algorithmic FP64 flops per line element of the Krylov direction pass
# (k_pred_line<HOM>): right-hand side 11, tridiagonal solve with stored factors 10,
# flux of the two faces 10.
HOM_FLOPS_PER_ELEM = 31
# Bytes a binary32 line pass with stored factors moves per line element: the five
# factor values read (1/den, a, c-hat, c-check, a-check) and the flux contribution
# written; the line's unknowns stay in shared memory.
LINE_BYTES_PER_ELEM_F32 = 5 * 4 + 4
# Bytes a Krylov-kernel launch (k_gmres, one cluster of 8 CTAs per instance) must move
# per cell: the e/o flux parts of all M angles of the pass before it (bulk type) and
# four double per-cell vectors (direction or iterate in, result out, two basis reads).
GMRES_BYTES_PER_CELL = lambda M, es: M * es + 4 * 8
# DRAM bytes per k_gmres<ARNOLDI> launch measured by ncu --set full (mean of two
# launches, cold cache) on the 1D slab workload in mixed precision.  The kernel has
# changed since (restart decision read before the CTAs' barriers); until the counters
# are taken again the line reports traffic as null and gives this figure as context.
GMRES_TRAFFIC_SLAB6_MIXED_EARLIER = 13.19e6
# DRAM bytes per k_gmres launch on the 1D slab workload in FP64, the mean over six
# consecutive launches of all modes (restart 18.4 MB, Arnoldi 3.8 and 3.7 MB, update 3.0
# and 1.0 MB, one launch whose instances had all stopped 0.07 MB; ncu dram__bytes_read.sum
# + dram__bytes_write.sum, profiles/ncu_gmres_fp64_slab6.md), taken with the kernel as it
# stands
GMRES_DRAM_BYTES_SLAB6_FP64 = 5.00e6
# Per-cell bytes the fused prediction solve must move besides the state: the binary64
# inputs it reads once (T^n, U^n, rho^n and the 16 coefficient arrays of the cell) and
# the outputs rho* and F* (20 x 8 B).
FUSED_BYTES_PER_CELL = 160
# dram__bytes_read.sum + dram__bytes_write.sum of one k_pred_fused launch on one 8192-cell,
# 64-direction slab run (ncu --set full; profiles/ncu_pred_fused_slab1.md), taken with the
# kernel as it stands; a slab launch carries one such instance per run
FUSED_DRAM_BYTES_SLAB_INSTANCE = 4.137216e6


def job_throughput(updates_per_step, steps, t_ms, world, dist=None, device="cuda"):
    """Whole-job throughput of weak-scaled replicas: every rank advanced its own copy of
    the workload by `steps` steps in t_ms (its own CUDA-event time); the job's time is
    the maximum over ranks and its work the updates of all ranks.  Returns (updates/s,
    max time in ms)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([t_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return updates_per_step * steps * world / (t_ms * 1e-3), t_ms


def workload_instances(name):
    from paper_1811_05579_gb300 import workloads as wl
    if name == "slab6":
        runs = wl.slab_1d_runs(steps=1)
        cfg = {"workload": "1d_slab_8192x64_sigma0_over_T3_6runs", "nx": 8192, "n_dir": 64,
               "runs": 6, "sigma0": [1, 10], "eps": [1, 1e-2, 1e-4], "dt": "0.5 dx"}
    elif name == "slab1":
        runs = [wl.slab_1d_runs(steps=1)[1]]
        cfg = {"workload": "1d_slab_8192x64_sigma0_1_eps_1e-2", "nx": 8192, "n_dir": 64, "runs": 1,
               "sigma0": 1, "eps": 1e-2, "dt": "0.5 dx"}
    elif name == "marshak128":
        runs = [wl.marshak_1d()]
        cfg = {"workload": "1d_marshak_128x16", "nx": 128, "n_dir": 16, "runs": 1}
    elif name == "batched256":
        runs = wl.batched_1d(256, steps=1)
        cfg = {"workload": "1d_batched_256_uneven", "runs": 256}
    else:
        raise SystemExit("unknown workload " + name)
    return runs, cfg


def specs_of(runs):
    from paper_1811_05579_gb300 import grte as G
    out = []
    for r in runs:
        M = r.n_dir // 2
        out.append(dict(nx=r.nx, n_angle=M, v=None, w=None, sigma=r.sigma, kind=r.kind, bc=r.bc,
                        bL=np.full(M, r.bL), bR=np.full(M, r.bR),
                        dt=r.dt, eps=r.eps, a=r.a, c=r.c, Cv=r.Cv))
    return out


def roofline_of(prof, runs, prec, hbm_peak, workload):
    """Roofline block of the dominant kernel (largest share of the profiled device time):
    algorithmic bytes (or flops) per launch over its average event-timed launch."""
    from paper_1811_05579_gb300 import grte as G
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    tot_prof = sum(v[0] for v in prof.values())
    nelem = sum(r.nx * (r.n_dir // 2) for r in runs)
    roof = None
    avg_s = dom_ms / dom_n * 1e-3
    if prec == G.FP64 and dom_name in ("pred_hom", "pred_full"):
        flops = HOM_FLOPS_PER_ELEM * nelem
        achieved = flops / avg_s / 1e9
        roof = {"kernel": "k_pred_line<%s,double>" % dom_name[5:].upper(), "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (fp64)", "frac": achieved / FP64_PEAK_GFLOPS,
                "peak_source": "nominal FP64 of the profiling recipe (1.25 TFLOP/s)",
                "traffic": None, "avg_launch_us": avg_s * 1e6, "launches": dom_n}
    elif dom_name in ("pred_hom", "pred_full", "pred_factor", "corr"):
        # binary32 line pass: bytes it must move per line element with stored factors
        # (4 factors + right-hand side/solution buffer write and read + flux out, 4 B each)
        byts = LINE_BYTES_PER_ELEM_F32 * nelem
        achieved = byts / avg_s / 1e9
        roof = {"kernel": "k_pred_line<%s,float>" % dom_name[5:].upper() if dom_name.startswith("pred") else "k_corr_line<float>",
                "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "traffic": None, "avg_launch_us": avg_s * 1e6, "launches": dom_n,
                "bytes_per_elem": LINE_BYTES_PER_ELEM_F32}
    elif dom_name == "pred_solve":
        # the fused prediction solve (one persistent cluster per instance): the bytes it
        # must move are the state read once (E, O in the bulk type) and per cell the
        # coefficient and vector traffic of the solve's inputs and outputs
        es = 8 if prec == G.FP64 else 4
        byts = sum(r.nx * (r.n_dir // 2) * 2 * es + r.nx * FUSED_BYTES_PER_CELL for r in runs)
        achieved = byts / avg_s / 1e9
        roof = {"kernel": "k_pred_fused (whole prediction solve per instance cluster)", "bound": "hbm",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "traffic": (FUSED_DRAM_BYTES_SLAB_INSTANCE * len(runs)
                            if workload in ("slab6", "slab1") and prec == G.MIXED else None),
                "traffic_source": "ncu dram bytes of one slab-run launch, times the runs in a launch",
                "algorithmic_bytes_per_launch": byts,
                "bytes_model": "state read once (2 x %d B per line element) + %d B per cell" % (es, FUSED_BYTES_PER_CELL),
                "avg_launch_us": avg_s * 1e6, "launches": dom_n,
                "note": "latency-bound: barrier and binary64 dependency chains of ~7 Krylov steps per launch"}
    elif dom_name == "gmres":
        es = 8 if prec == G.FP64 else 4
        M = runs[0].n_dir // 2
        byts = sum(r.nx for r in runs) * GMRES_BYTES_PER_CELL(M, es)
        achieved = byts / avg_s / 1e9
        earlier = GMRES_TRAFFIC_SLAB6_MIXED_EARLIER if (workload == "slab6" and prec == G.MIXED) else None
        roof = {"kernel": "k_gmres (all modes; Arnoldi step dominant)", "bound": "hbm", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "traffic": GMRES_DRAM_BYTES_SLAB6_FP64 if (workload == "slab6" and prec == G.FP64) else None,
                "traffic_source": "ncu dram bytes, mean of six launches of all modes",
                "traffic_before_last_kernel_change": earlier,
                "avg_launch_us": avg_s * 1e6, "launches": dom_n, "bytes_per_cell": GMRES_BYTES_PER_CELL(M, es),
                "bytes_model": "achieved and frac from the byte model: M x %d B flux parts + 4 x 8 B per cell" % es}
    else:
        roof = {"kernel": dom_name, "bound": "alu", "achieved": None, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s (fp64)", "frac": None, "traffic": None,
                "avg_launch_us": avg_s * 1e6, "launches": dom_n}
    return roof, dom_name


def mlp_throughput(n_inf=1 << 20, n_train=1 << 17, epochs=3, batch=4096):
    """The learned guess's network on the tensor cores: inference samples/s on device
    arrays (CUDA events over 10 calls after 3) and training samples/s (grte_mlp_train:
    forward, backward, Adam per batch; wall clock over `epochs` epochs, the host shuffle
    and the per-epoch upload included)."""
    import torch
    from paper_1811_05579_gb300 import grte as G
    m = G.MLP(seed=1)
    rng = np.random.default_rng(7)
    X = torch.tensor(rng.standard_normal((n_inf, 6)), dtype=torch.float32, device="cuda")
    y = torch.empty(n_inf, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        m.forward_device(X.data_ptr(), n_inf, y.data_ptr(), stream.cuda_stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        m.forward_device(X.data_ptr(), n_inf, y.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    inf = 10 * n_inf / (e0.elapsed_time(e1) * 1e-3)
    Xt = rng.standard_normal((n_train, 6)).astype(np.float32)
    Yt = rng.standard_normal(n_train).astype(np.float32)
    m.train(Xt, Yt, epochs=1, batch=batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.train(Xt, Yt, epochs=epochs, batch=batch)
    tr = n_train * epochs / (time.perf_counter() - t0)
    m.close()
    return {"inference_samples_per_s": inf, "inference_batch": n_inf,
            "training_samples_per_s": tr, "training_batch": batch, "training_samples": n_train,
            "kernels": "mma.sync m16n8k16 BF16 -> FP32 (forward, backward deltas, weight gradients)"}


def sub_result(name, steps, warmup, sequential=False):
    """A further workload on the same GPU: the mixed form (the library's default solve)
    and the plain FP64 form, each timed with CUDA events over `steps` steps after
    `warmup`, the T error of the mixed form against FP64 after the same steps, and one
    step of each from the FP64 state reached; with `sequential`, the instances also
    advanced one handle each, one after the other."""
    import torch
    from paper_1811_05579_gb300 import grte as G
    runs, cfg = workload_instances(name)
    specs = specs_of(runs)
    ups = sum(r.nx * r.n_dir for r in runs)
    stream = torch.cuda.current_stream()
    out = {"config": cfg, "steps": steps, "warmup": warmup}
    hs = {}
    for key, prec in (("mixed", G.MIXED), ("fp64", G.FP64)):
        h = G.Grte(specs, precision=prec, stream=stream.cuda_stream)
        for i, r in enumerate(runs):
            h.set_state(i, r.T0)
        for _ in range(warmup):
            h.step(1)
        h.sync(allow=ALLOW1D)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[key] = {"value": ups / (ms * 1e-3), "ms_per_step": ms}
        hs[key] = h
    errs = []
    for i in range(len(runs)):
        a_, b_ = hs["mixed"].T(i, allow=ALLOW1D), hs["fp64"].T(i, allow=ALLOW1D)
        errs.append(float(np.max(np.abs(a_ - b_) / np.maximum(np.abs(b_), 1e-300))))
    out["t_max_rel_err_trajectory"] = max(errs)
    snap = [(hs["fp64"].T(i, allow=ALLOW1D), hs["fp64"].E(i, allow=ALLOW1D), hs["fp64"].O(i, allow=ALLOW1D))
            for i in range(len(runs))]
    one = {}
    for key, prec in (("mixed", G.MIXED), ("fp64", G.FP64)):
        h = G.Grte(specs, precision=prec, stream=stream.cuda_stream)
        for i, (T_, E_, O_) in enumerate(snap):
            h.set_state(i, T_, E_, O_)
        h.step(1)
        one[key] = [h.T(i, allow=ALLOW1D) for i in range(len(runs))]
        h.close()
    out["t_max_rel_err_one_step"] = max(float(np.max(np.abs(a_ - b_) / np.maximum(np.abs(b_), 1e-300)))
                                        for a_, b_ in zip(one["mixed"], one["fp64"]))
    for h in hs.values():
        h.close()
    if sequential:
        hl = [G.Grte([sp], precision=G.MIXED, stream=stream.cuda_stream) for sp in specs]
        for hh, r in zip(hl, runs):
            hh.set_state(0, r.T0)
            hh.step(1)
        ks = 2
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ks):
            for hh in hl:
                hh.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / ks
        out["sequential_mixed"] = {"value": ups / (ms * 1e-3), "ms_per_step": ms, "handles": len(hl), "steps": ks}
        for hh in hl:
            hh.close()
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from paper_1811_05579_gb300 import workloads as wl
from oracle import grte1d as og
from oracle.quadrature import gauss_legendre_half
runs, _ = None, None
r = wl.slab_1d_runs(steps=1)[1]
v, w = gauss_legendre_half(r.n_dir)
P = og.Problem(N=r.nx, v=v, w=w, sig=r.sigma, eps=r.eps, dt=r.dt, kind="t3",
               bL=np.ones(v.size), bR=np.zeros(v.size))
S = og.equilibrium_state(P, r.T0)
S = og.step(P, S)          # untimed warm-up step
n = {nsteps}
t0 = time.perf_counter()
for _ in range(n):
    S = og.step(P, S)
dt = time.perf_counter() - t0
print(json.dumps({{"updates": n * r.nx * r.n_dir, "seconds": dt, "steps": n}}))
"""


def cpu_baseline(nsteps=3):
    """The oracle as it stands, single-threaded, on one of the six runs
    (sigma0 = 1, eps = 1e-2; 8192 cells x 64 directions) for nsteps steps."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", CPU_SNIPPET.format(root=ROOT, nsteps=nsteps)],
                         capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(), "kind": "oracle",
                "sample": "failed: " + out.stderr.strip()[-200:]}
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": d["updates"] / d["seconds"], "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d steps of one run (sigma0=1, eps=1e-2, 8192 cells x 64 dirs), %.1f s, 1 thread"
                      % (d["steps"], d["seconds"])}


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(nsteps=max(1, min(args.steps, 3)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# statuses a 1D step may end with and still be measured: 5 (cells whose correction
# right-hand side reached R <= 0) and 4 (a prediction solve that ran its restart cycles
# without meeting the tolerance; the slab runs with sigma_0 = 1, eps <= 1e-2 are unstable
# at dt = dx/2 and their mixed-precision solves can end so)
ALLOW1D = (4, 5)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="slab6",
                    choices=["slab6", "slab1", "marshak128", "batched256", "checker2d", "lognormal2d"])
    ap.add_argument("--n2d", type=int, default=None,
                    help="cells per axis of the 2D workloads (checker2d: 128, lognormal2d: 512)")
    ap.add_argument("--newton-start", default="bound", choices=["bound", "previous", "learned"],
                    help="2D: Newton's starting point (learned: a network trained first on small 2D runs)")
    ap.add_argument("--krylov-restart", type=int, default=None,
                    help="2D: GMRES restart length (checker2d: 30, lognormal2d: 60)")
    ap.add_argument("--krylov-maxcycles", type=int, default=None,
                    help="2D: GMRES restart cycles per solve (checker2d: 30, lognormal2d: 60)")
    ap.add_argument("--compare-starts", action="store_true",
                    help="2D: also run the other Newton starts from the same state and report their counts")
    ap.add_argument("--prec2d", default="block", choices=["block", "multigrid", "corr-mg", "multigrid+corr-mg"],
                    help="2D preconditioners: prediction per-cell block (+ multigrid on rho: 'multigrid'); "
                         "correction per-cell diagonal (+ per-pair multigrid: 'corr-mg')")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--line-threads", type=int, default=0, choices=[0, 256, 512, 1024],
                    help="threads per line solve (0: the library's autotuner)")
    ap.add_argument("--sequential-compare", action="store_true",
                    help="also time the same instances advanced one handle at a time")
    ap.add_argument("--no-sub-results", action="store_true",
                    help="slab workload: skip the batched 256-instance and 128-cell Marshak sub-results")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload in ("checker2d", "lognormal2d"):
        if args.n2d is None:
            # 1024^2 random-smooth stops with ENONCONV in the correction substep (its Jacobi
            # preconditioner); 512^2 is the largest size measured to converge
            args.n2d = 128 if args.workload == "checker2d" else 512
        if args.krylov_restart is None:
            args.krylov_restart = 30 if args.workload == "checker2d" else 60
        if args.krylov_maxcycles is None:
            args.krylov_maxcycles = 30 if args.workload == "checker2d" else 60
        if args.impl == "reference":
            if int(os.environ.get("RANK", "0")) == 0:
                cb = cpu_baseline_2d(workload=args.workload)
                print(json.dumps({"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
                                  "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                                  "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                                  "dtype": "f64", "data": "synthetic",
                                  "config": {"workload": workload_name_2d(args.workload, args.n2d)},
                                  "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT,
                                                              "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return
        return run_2d(args)
    runs, cfg = workload_instances(args.workload)
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1811_05579_gb300 import grte as G

    stream = torch.cuda.current_stream()
    specs = specs_of(runs)
    prec = G.MIXED if args.precision == "mixed" else G.FP64
    h = G.Grte(specs, precision=prec, stream=stream.cuda_stream, line_threads=args.line_threads)
    for i, r in enumerate(runs):
        h.set_state(i, r.T0)
    updates_per_step = sum(r.nx * r.n_dir for r in runs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        h.step(1)
    h.sync(allow=ALLOW1D)
    tune = h.tuning()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    kry_its = 0
    kry_cycles = 0
    for k in range(args.steps):
        flush.zero_()                 # L2 flushed between timed steps (not timed)
        starts[k].record(stream)
        h.step(1)                     # one CUDA graph launch per step (after the first step)
        ends[k].record(stream)
        launches += h.last_launches()
        st = h.stats(allow=ALLOW1D)
        kry_its += st["krylov_iters"]
        kry_cycles += st["krylov_cycles"]
    barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = float(np.sum(step_ms))
    # per-kernel times: a graph hides kernel boundaries from events, so the same
    # workload continues for a few eager steps with an event pair around every launch
    # on the handle's stream
    kp = min(args.steps, 5)
    h.profile_begin(G.KERNELS)
    for _ in range(kp):
        flush.zero_()
        h.step(1)
    prof = h.profile_end()
    torch.cuda.synchronize()
    value, t_ms = job_throughput(updates_per_step, args.steps, t_ms, world, dist, "cuda")

    # end to end through the public API with host buffers: state in (H2D), one step,
    # temperature out (D2H), timed on the host clock with the stream synchronised
    host_state = []
    for i, r in enumerate(runs):
        host_state.append((h.T(i, allow=ALLOW1D), h.E(i, allow=ALLOW1D), h.O(i, allow=ALLOW1D)))
    h2d = sum(T.nbytes + E.nbytes + O.nbytes for T, E, O in host_state)
    d2h = sum(T.nbytes for T, _, _ in host_state)
    ke = min(args.steps, 5)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        for i, (T, E, O) in enumerate(host_state):
            h.set_state(i, T, E, O)
        h.step(1)
        for i in range(len(runs)):
            h.T(i, allow=ALLOW1D)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    e2e_val = updates_per_step * ke / te

    # the same workload in FP64 (the plain form): timed the same way, and the
    # temperature error of the benchmarked form against it after the same steps
    cmp = None
    if prec == G.MIXED and not args.no_fp64_compare:
        hd = G.Grte(specs, precision=G.FP64, stream=stream.cuda_stream)
        for i, r in enumerate(runs):
            hd.set_state(i, r.T0)
        hm = G.Grte(specs, precision=prec, stream=stream.cuda_stream)
        for i, r in enumerate(runs):
            hm.set_state(i, r.T0)
        for _ in range(args.warmup):
            hd.step(1)
            hm.step(1)
        t64 = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hd.step(1)
            e1.record(stream)
            hm.step(1)
            torch.cuda.synchronize()
            t64 += e0.elapsed_time(e1)
        errs = []
        for i in range(len(runs)):
            a_ = hm.T(i, allow=ALLOW1D)
            b_ = hd.T(i, allow=ALLOW1D)
            errs.append(float(np.max(np.abs(a_ - b_) / np.maximum(np.abs(b_), 1e-300))))
        # one step of each form from the FP64 state reached: the error of the precision
        # itself (over a trajectory an unstable run amplifies it step by step)
        snap = [(hd.T(i, allow=ALLOW1D), hd.E(i, allow=ALLOW1D), hd.O(i, allow=ALLOW1D)) for i in range(len(runs))]
        h1 = G.Grte(specs, precision=prec, stream=stream.cuda_stream)
        h2 = G.Grte(specs, precision=G.FP64, stream=stream.cuda_stream)
        for i, (T_, E_, O_) in enumerate(snap):
            h1.set_state(i, T_, E_, O_)
            h2.set_state(i, T_, E_, O_)
        h1.step(1)
        h2.step(1)
        errs1 = []
        for i in range(len(runs)):
            a_ = h1.T(i, allow=ALLOW1D)
            b_ = h2.T(i, allow=ALLOW1D)
            errs1.append(float(np.max(np.abs(a_ - b_) / np.maximum(np.abs(b_), 1e-300))))
        h1.close()
        h2.close()
        cmp = {"fp64_value": updates_per_step * args.steps / (t64 * 1e-3), "fp64_ms_per_step": t64 / args.steps,
               "t_max_rel_err_one_step": max(errs1), "t_rel_err_one_step_per_run": errs1,
               "t_max_rel_err_trajectory": max(errs), "t_rel_err_trajectory_per_run": errs,
               "steps_compared": args.warmup + args.steps}
        # the FP64 form's own roofline: per-kernel event pairs over a few eager steps
        hd.profile_begin(G.KERNELS)
        for _ in range(min(args.steps, 3)):
            flush.zero_()
            hd.step(1)
        prof64 = hd.profile_end()
        torch.cuda.synchronize()
        peak = 6800.0
        try:
            peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        except Exception:
            pass
        cmp["fp64_roofline"] = roofline_of(prof64, runs, G.FP64, peak, args.workload)[0]
        cmp["fp64_kernel_share"] = {k: round(v[0] / sum(x[0] for x in prof64.values()), 4)
                                    for k, v in sorted(prof64.items())}
        hd.close()
        hm.close()

    # the same instances, one handle each, stepped one after the other
    seq = None
    if args.sequential_compare:
        hs = [G.Grte([sp], precision=prec, stream=stream.cuda_stream) for sp in specs]
        for hh, r in zip(hs, runs):
            hh.set_state(0, r.T0)
        for hh in hs:
            hh.step(1)
        ks = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ks):
            for hh in hs:
                hh.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        tseq = e0.elapsed_time(e1)
        seq = {"value": updates_per_step * ks / (tseq * 1e-3), "ms_per_step": tseq / ks, "steps": ks,
               "handles": len(hs)}
        for hh in hs:
            hh.close()
    hbm_peak = 6800.0
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    roof, dom_name = roofline_of(prof, runs, prec, hbm_peak, args.workload)
    tot_prof = sum(v[0] for v in prof.values())
    step_s = t_ms * 1e-3 / args.steps
    bpu = 24 if prec == G.FP64 else 12
    h_mode = ("one CUDA graph launch per step: the prediction solve is one persistent cluster kernel per "
              "instance" if "pred_solve" in prof else
              "one CUDA graph launch per step (Krylov loop under device-side conditional nodes)")
    hbm_alg = updates_per_step * bpu / step_s / 1e9    # state read twice, written once per update

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == G.FP64 else "f32 bulk / f64 per-cell, Newton, sums",
                "data": "synthetic (seeded; no dataset)",
                "config": dict(cfg, l2="flushed between timed steps (flush not timed)", precision=args.precision,
                               parallelism="replicas" if world > 1 else "single"),
                "gpu_launches": launches,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "roofline": roof,
                "step_hbm_roofline": {"algorithmic_bytes_per_update": bpu, "achieved_gbs": hbm_alg,
                                      "peak_gbs": hbm_peak, "frac": hbm_alg / hbm_peak},
                "step_mode": h_mode,
                "kernel_share": {k: round(v[0] / tot_prof, 4) for k, v in sorted(prof.items())},
                "kernel_profile": "event pairs around every launch over %d further eager steps of the same workload" % kp,
                "krylov_iters_per_step": kry_its / args.steps / len(runs),
                "krylov_cycles_per_step": kry_cycles / args.steps,
                "line_tuning": {"threads": tune[0], "candidates_ms": tune[1], "smem": bool(h.stats(allow=ALLOW1D)["line_smem"])},
                "statuses_seen": [n_ for b_, n_ in ((4, "ENONCONV"), (5, "R<=0 cells"))
                                  if h.stats(allow=ALLOW1D)["status_flags"] & (1 << b_)],
                "clocks": clk}
        if cmp is not None:
            line["vs_fp64"] = cmp
        if args.workload == "slab6" and prec == G.MIXED and not args.no_sub_results and world == 1:
            line["sub_results"] = {"batched256": sub_result("batched256", 5, 3, sequential=True),
                                   "marshak128": sub_result("marshak128", 125, 3),
                                   "learned_guess_mlp": mlp_throughput()}
        if seq is not None:
            line["sequential"] = seq
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()


def dt_2d(n):
    """Time step of the 2D workloads (their configurations give none): the paper's Table
    stability3 (the Marshak wave under a hot wall) lowers the stable C = dt/dx from 0.5 at
    dx = 1/25 to 0.03 at 1/400, about C = 12.5 dx; dt = min(0.5 dx, 12.5 dx^2).  At
    dt = 0.5 dx the 2D runs (and the oracle: a 32^2 checkerboard reaches T = 4.8 under a
    unit inflow within 5 steps) empty cells and overshoot."""
    return min(0.5 / n, 12.5 / (n * n))


def checker2d_inputs(n, blocks=8):
    """2D checkerboard slab: sigma_0 = 1 on the 'black' and 100 on the 'white' blocks of a
    blocks x blocks board (block (0, 0) black), times 1/T^3; T_in = 1e-2; eps = 1e-3;
    inflow a c 1^4 on x = 0, vacuum on the other walls; dt = dt_2d(n); S8 (20 pairs)."""
    i = np.arange(n) // max(n // blocks, 1)
    sig = np.where(((i[None, :] + i[:, None]) % 2) == 0, 1.0, 100.0)
    return sig, np.full(n * n, 1e-2), dt_2d(n), 1e-3


def lognormal2d_inputs(n):
    """2D random-smooth slab: sigma_0 = exp(g), g an iid N(0, 1) field smoothed by a
    Gaussian of standard deviation 8 cells (wrapped, separable) and renormalised to unit
    variance, times 1/T^3; T_in = 1e-2; eps = 1e-4; inflow a c 1^4 on x = 0, vacuum on
    the other walls; dt = dt_2d(n); S8 (20 pairs)."""
    from paper_1811_05579_gb300 import workloads as wl
    sig = wl.lognormal_sigma_2d(n, seed=wl.BASE_SEED + 5, sd_cells=8.0)
    return sig, np.full(n * n, 1e-2), dt_2d(n), 1e-4


def inputs_2d(workload, n):
    return checker2d_inputs(n) if workload == "checker2d" else lognormal2d_inputs(n)


def workload_name_2d(workload, n):
    return ("2d_checkerboard_%dx%d_s8" if workload == "checker2d" else "2d_lognormal_%dx%d_s8") % (n, n)


def cpu_baseline_2d(n=16, nsteps=8, workload="checker2d"):
    """The 2D oracle as it stands, one thread, on the same geometry at n x n."""
    code = f"""
import os, sys, time, json
os.environ["OMP_NUM_THREADS"] = "1"; os.environ["OPENBLAS_NUM_THREADS"] = "1"
sys.path.insert(0, {ROOT!r})
import numpy as np
import bench
from oracle import grte2d as o2
from oracle.quadrature import s8_pairs_2d
sig, T0, dt, eps = bench.inputs_2d({workload!r}, {n})
mu, eta, w = s8_pairs_2d()
P = o2.Problem2D(Nx={n}, Ny={n}, mu=mu, eta=eta, w=w, sig=sig, eps=eps, dt=dt, kind="t3", bx0=1.0)
S = o2.equilibrium_state(P, T0)
t = time.perf_counter()
for _ in range({nsteps}):
    S = o2.step(P, S)
dt_ = time.perf_counter() - t
print(json.dumps({{"updates": {n} * {n} * 40 * {nsteps}, "seconds": dt_}}))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["updates"] / d["seconds"], "unit": UNIT, "cores": 1, "host_nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d step(s) of the same geometry at %dx%d (sparse LU), %.1f s, 1 thread" % (nsteps, n, n, d["seconds"])}


def train_guess_2d(G, stream):
    """A network for the learned Newton start, trained on the GPU on the scheme's own
    (features -> log10 T^{n+1}/T^n) pairs logged by small 2D runs: checkerboards with
    per-run sigma_0 values (log-uniform in [10^-0.5, 1] and [10, 100]) and log-normal
    fields of other seeds, 24^2-56^2, eps 1e-3 and 1e-4, 25 steps each."""
    from paper_1811_05579_gb300 import workloads as wl
    runs = []
    for r, n in enumerate((24, 32, 40, 56)):
        u = wl.SplitMix64(wl.BASE_SEED + 100 + r).uniform(2)
        runs.append((n, wl.checkerboard_sigma_2d(n, lo=10 ** (-0.5 + 0.5 * u[0]), hi=10 ** (1.0 + u[1])),
                     1e-3 if r % 2 == 0 else 1e-4, 41 + r))
    for r, n in enumerate((32, 40)):
        runs.append((n, wl.lognormal_sigma_2d(n, seed=wl.BASE_SEED + 11 + r, sd_cells=3.0), 1e-4, 51 + r))
    Xs, Ys = [], []
    t0 = time.perf_counter()
    for n, sig, eps, seed in runs:
        h = G.Grte2D(n, n, sig, dt_2d(n), eps, kind=G.SIGMA_T3, b_x0=1.0, stream=stream.cuda_stream)
        h.set_state(1e-2 * (1.0 + 0.5 * wl.SplitMix64(seed).uniform(n * n)))
        h.set_sample_logging(True)
        for _ in range(25):
            h.step(1, allow=(5,))
            X, y = h.newton_samples()
            keep = np.all(np.isfinite(X), axis=1) & (X[:, 0] > -30) & (np.abs(X[:, 2]) < 30)
            Xs.append(X[keep])
            Ys.append(y[keep])
        h.close()
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    m = G.MLP(seed=1)
    m.set_norm(X.mean(0), np.maximum(X.std(0), 0.1), float(Y.mean()), float(Y.std() + 1e-6))
    loss = m.train(X, Y, epochs=30, batch=256, lr=1e-3, seed=3)
    return m, {"samples": int(X.shape[0]), "standardised_mse": float(loss), "seconds": time.perf_counter() - t0}


def run_2d(args):
    """The 2D path (grte2d_*) on the checkerboard or the random-smooth workload at n2d x n2d."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:   # weak-scaled replicas: each rank its own copy, max time over ranks
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1811_05579_gb300 import grte as G
    n = args.n2d
    sig, T0, dt, eps = inputs_2d(args.workload, n)
    stream = torch.cuda.current_stream()
    net, training = None, None
    if args.newton_start == "learned" or args.compare_starts:
        net, training = train_guess_2d(G, stream)
    prec = ((G.PREC2D_MULTIGRID if args.prec2d.startswith("multigrid") else G.PREC2D_BLOCK) |
            (G.PREC2D_CORR_MG if args.prec2d.endswith("corr-mg") else 0))
    precision = G.MIXED if args.precision == "mixed" else G.FP64
    # cells reaching R <= 0, and solves that stop at their cycle limit (both reported in
    # statuses_seen)
    allow = (4, 5)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    snap = {}
    seen_codes = set()   # statuses the timed steps returned

    def timed(precision_, clocks=None, start=args.newton_start):
        h_ = G.Grte2D(n, n, sig, dt, eps, kind=G.SIGMA_T3, b_x0=1.0, stream=stream.cuda_stream, prec=prec,
                      precision=precision_, krylov_restart=args.krylov_restart,
                      krylov_maxcycles=args.krylov_maxcycles)
        if start == "learned":
            h_.set_guess(net)
        elif start == "previous":
            h_.set_newton_start(G.START_PREVIOUS)
        h_.set_state(T0)
        for _ in range(args.warmup):
            h_.step(1, allow=allow)
        if clocks:   # the state the timed steps start from (for the end-to-end replay)
            snap["state"] = (h_.T(allow), h_.E(allow), h_.O(allow))
        if clocks and dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        t, it = 0.0, [0, 0, 0, 0.0, 0]
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            seen_codes.add(h_.step(1, allow=allow))
            e1.record(stream)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1)
            st = h_.stats(allow=allow)
            it[0] += st["krylov_iters"]
            it[1] += st["krylov_iters_corr"]
            it[2] += st["krylov_iters_mg"]
            it[3] += st["newton_iters_mean"] / args.steps
            it[4] += st["launches"]
        if clocks and dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        return h_, t, it

    clocks = ClockSampler(local)
    h, t_ms, (its, its_corr, its_mg, newton_mean, launches) = timed(precision, clocks)
    clk = clocks.stop()
    starts = None
    if args.compare_starts:
        starts = {args.newton_start: {"ms_per_step": t_ms / args.steps, "newton_iters_per_cell": newton_mean}}
        for other in ("bound", "previous", "learned"):
            if other != args.newton_start:
                h2, t2, it2 = timed(precision, start=other)
                starts[other] = {"ms_per_step": t2 / args.steps, "newton_iters_per_cell": it2[3],
                                 "t_max_rel_diff": float(np.max(np.abs(h2.T(allow) - h.T(allow)) /
                                                                np.maximum(np.abs(h.T(allow)), 1e-300)))}
                h2.close()
    vs_fp64 = None
    if precision == G.MIXED and not args.no_fp64_compare:
        h64, t64, _ = timed(G.FP64)
        Tm, T64 = h.T(allow), h64.T(allow)
        vs_fp64 = {"fp64_ms_per_step": t64 / args.steps, "fp64_value": n * n * 40 * args.steps / (t64 * 1e-3),
                   "t_max_rel_err_vs_fp64": float(np.max(np.abs(Tm - T64) / np.maximum(np.abs(T64), 1e-300))),
                   "steps_compared": args.warmup + args.steps}
        h64.close()
    upd = n * n * 40
    value, t_ms = job_throughput(upd, args.steps, t_ms, world, dist)
    # end to end through the public API with host buffers: the same K steps from the same
    # state, each one copying the whole state (T, E, O) in, stepping and copying it out
    T, E, O = snap["state"]
    torch.cuda.synchronize()
    t_e2e = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h.set_state(T, E, O)
        h.step(1, allow=allow)
        T, E, O = h.T(allow), h.E(allow), h.O(allow)
        t_e2e += time.perf_counter() - t0
    e2e = upd * args.steps / t_e2e
    hbm_peak = 6800.0
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    step_s = t_ms * 1e-3 / args.steps
    ach = upd * 24 / step_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 Krylov cycles / f64 residual, Newton, sums" if precision == G.MIXED else "f64",
            "data": "synthetic (seeded; no dataset)",
            "config": {"workload": workload_name_2d(args.workload, n), "n": n, "pairs": 20, "eps": eps,
                       "precision": args.precision,
                       "sigma0": [1, 100] if args.workload == "checker2d" else "exp(N(0,1) smoothed 8 cells)",
                       "dt": "min(0.5 dx, 12.5 dx^2) = %.3g" % dt, "T_in": 1e-2, "prec2d": args.prec2d,
                       "newton_start": args.newton_start, "krylov_restart": args.krylov_restart,
                       "krylov_maxcycles": args.krylov_maxcycles,
                       "l2": "flushed between timed steps (flush not timed)", "parallelism": "single"},
            "gpu_launches": launches,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(T.nbytes + E.nbytes + O.nbytes),
                    "d2h_bytes_per_step": int(T.nbytes + E.nbytes + O.nbytes),
                    "note": "replays the timed steps from the same state; L2 not flushed"},
            "roofline": {"kernel": "2D step (all kernels)", "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                         "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None,
                         "note": "24 B per cell-angle update over the step time"},
            "statuses_seen": [n_ for b_, n_ in ((4, "ENONCONV"), (5, "R<=0 cells")) if b_ in seen_codes],
            "krylov_iters_per_step": its / args.steps, "krylov_iters_corr_per_step": its_corr / args.steps,
            "krylov_iters_mg_per_step": its_mg / args.steps, "vs_fp64": vs_fp64,
            "newton_iters_per_cell": newton_mean, "newton_starts": starts, "guess_training": training,
            "status_flags": h.stats(allow=allow)["status_flags"],
            "clocks": clk}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_2d(workload=args.workload)
    if rank == 0:
        print(json.dumps(line))
    h.close()
    if net is not None:
        net.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
