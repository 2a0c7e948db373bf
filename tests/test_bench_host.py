"""Host logic of bench.py, without a GPU: the reference arm (the CPU oracle)
prints one JSON line with the keys the benchmark line carries and only rank 0
prints it; the roofline arithmetic of the dominant kernel; the clock sample
summary."""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def _run_reference(env_extra):
    env = dict(os.environ, OMP_NUM_THREADS="4", **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "vortex64", "--steps", "2", "--warmup", "1"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_line(orc):
    r = _run_reference({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "cell-updates/s per S2O4 step"
    assert d["unit"] == "cell-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "vortex64"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 4 and cb["sample"]
    # value = cells x steps / time
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - 64 * 64) < 1e-6 * 64 * 64


def test_reference_arm_other_ranks_print_nothing(orc):
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_roofline_dominant_kernel(bench):
    n = 128 ** 3
    prof = {"recon": (10, 259.0), "flux": (10, 1028.0), "update": (10, 30.8), "dt": (5, 0.35)}
    r = bench.roofline(prof, bench.WORKLOADS["tgv128"], n, 0, True)
    assert r["kernel"] == "flux" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    units = n * 3 * 4                       # 12 face Gauss points owned per cell in 3-D
    assert r["units_per_launch"] == units
    assert r["flops_per_launch"] == pytest.approx(2919.0 * units)  # algorithmic count
    assert r["achieved"] == pytest.approx(2919.0 * units / 0.1028 / 1e12)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_executed"] == pytest.approx(3.616e3 * units / 0.1028 / 1e12 / r["peak"])
    assert r["traffic"] == pytest.approx((1.0084e9 + 0.7103e9) * 8)   # 64^3 capture scaled to 128^3


def test_roofline_uncounted_kernel(bench):
    """a dominant kernel without a counted flop figure reports no fraction"""
    r = bench.roofline({"recon": (2, 100.0), "flux": (2, 50.0)}, bench.WORKLOADS["tgv128"], 128 ** 3, 0, True)
    assert r["kernel"] == "recon" and r["achieved"] is None and r["frac"] is None and "note" in r


def test_roofline_fp32_flux(bench):
    n = 64 * 64 * 64
    r = bench.roofline({"flux": (4, 4.0), "update": (4, 1.0)}, bench.WORKLOADS["tgv64"], n, 1, True)
    assert r["kernel"] == "flux"
    assert r["flops_per_launch"] == pytest.approx(2919.0 * n * 12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["frac_executed"] == pytest.approx(3.395e3 * n * 12 / 1e-3 / 1e12 / r["peak"])


def test_step_hbm_share(bench):
    """the step-level HBM share counts six FP64 state transfers per cell
    (SURVEY-style algorithmic bytes: 3.84 KB per 3-D cell, 1.34 KB in 2-D)"""
    r = bench.step_hbm(2097152, 3, 135.0, 6691.1)
    assert r["algorithmic_bytes_per_cell"] == 6 * 640
    assert r["achieved_gbs"] == pytest.approx(2097152 * 3840 / 0.135 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 6691.1)
    assert bench.step_hbm(4096, 2, 1.0, None)["algorithmic_bytes_per_cell"] == 6 * 224
    assert bench.step_hbm(4096, 2, 1.0, None)["frac"] is None
