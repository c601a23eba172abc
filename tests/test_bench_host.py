"""Host logic of bench.py that needs no GPU: the 2D workload inputs and the reference arm
(the oracle timed on the host), whose JSON line the driver reads."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_checkerboard_inputs():
    sig, T0, dt, eps = bench.inputs_2d("checker2d", 64)
    assert sig.shape == (64, 64) and T0.shape == (64 * 64,)
    assert set(np.unique(sig)) == {1.0, 100.0}
    assert sig[0, 0] == 1.0 and sig[0, 8] == 100.0 and sig[8, 8] == 1.0   # 8 x 8 board, block (0, 0) black
    # dt = min(0.5 dx, 12.5 dx^2), the trend of Table stability3 (C = 12.5 dx)
    assert np.all(T0 == 1e-2) and dt == min(0.5 / 64, 12.5 / 64 ** 2) and eps == 1e-3
    assert abs(bench.dt_2d(512) * 512 - 12.5 / 512) < 1e-15 and bench.dt_2d(16) == 0.5 / 16
    assert bench.workload_name_2d("checker2d", 64) == "2d_checkerboard_64x64_s8"


def test_random_smooth_inputs():
    sig, T0, dt, eps = bench.inputs_2d("lognormal2d", 96)
    g = np.log(sig)
    assert sig.shape == (96, 96) and np.all(sig > 0)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    assert np.all(T0 == 1e-2) and dt == min(0.5 / 96, 12.5 / 96 ** 2) and eps == 1e-4
    # seeded: the same field every time
    assert np.array_equal(sig, bench.inputs_2d("lognormal2d", 96)[0])
    assert bench.workload_name_2d("lognormal2d", 96) == "2d_lognormal_96x96_s8"


def test_reference_arm_line_for_the_random_smooth_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "lognormal2d", "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "2d_lognormal_512x512_s8"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_roofline_blocks_carry_measured_traffic_and_label_models():
    """The dominant kernel's roofline block: achieved = algorithmic bytes per launch /
    average launch time; traffic = the ncu DRAM bytes where a capture of the current kernel
    exists (the one-kernel solve per slab run times the runs; k_gmres in FP64 on the slab),
    and every figure that comes from a byte model says so."""
    from paper_1811_05579_gb300 import grte as G
    runs, _ = bench.workload_instances("slab6")
    r, name = bench.roofline_of({"pred_solve": (10.0, 10)}, runs, G.MIXED, 6689.5, "slab6")
    assert name == "pred_solve" and r["bound"] == "hbm"
    assert r["traffic"] == bench.FUSED_DRAM_BYTES_SLAB_INSTANCE * len(runs)
    nx = sum(q.nx for q in runs)
    nel = sum(q.nx * (q.n_dir // 2) for q in runs)
    assert r["algorithmic_bytes_per_launch"] == 2 * 4 * nel + bench.FUSED_BYTES_PER_CELL * nx
    assert abs(r["achieved"] - r["algorithmic_bytes_per_launch"] / 1e-3 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6689.5) < 1e-15
    r, name = bench.roofline_of({"gmres": (10.0, 100), "pred_hom": (5.0, 100)}, runs, G.FP64, 6689.5, "slab6")
    assert name == "gmres" and r["traffic"] == bench.GMRES_DRAM_BYTES_SLAB6_FP64
    assert "byte model" in r["bytes_model"]
    r, _ = bench.roofline_of({"gmres": (10.0, 100)}, runs, G.MIXED, 6689.5, "slab6")
    assert r["traffic"] is None   # no capture of the mixed k_gmres since it changed
