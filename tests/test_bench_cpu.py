"""The benchmark's CPU-side contract: the reference arm (the oracle timed on the host
cores) prints one JSON line with the keys the driver reads, and the CPU baseline sizes
its ray sample to the requested time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["unit"] == "ray segments/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("large")
    assert "refill" in d["cpu_baseline"]["sample"] and d["cpu_baseline"]["cpu_model"]


def test_cpu_baseline_scales_the_sample_to_the_target():
    sys.path.insert(0, ROOT)
    import bench
    # the medium workload keeps this test short (the default large one has its own
    # reference-arm test above)
    wl, bench.WORKLOAD_NAME, bench.SCENE = bench.WORKLOADS["medium"]
    bench.WORKLOAD.clear()
    bench.WORKLOAD.update(wl)
    out = bench.cpu_baseline(target_s=2.0, single_s=1.0)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == (os.cpu_count() or 1)
    assert out["cpu_model"] and out["single_thread"]["cores"] == 1 and out["single_thread"]["value"] > 0
    for o, target in ((out, 2.0), (out["single_thread"], 1.0)):
        rays = int(o["sample"].split(" ")[0])
        wall = float(o["sample"].rsplit(", ", 1)[1].split(" ")[0])
        # grown past the 20-ray probe until the sample takes about the target (or the workload)
        assert rays > 20 and (wall >= 0.5 * target or rays == bench.WORKLOAD["num_rays"])


def test_reference_arm_at_the_papers_operating_point():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "paper", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"].startswith("paper operating point") and d["config"]["sample_rays_per_step"] == 50


def test_reference_arm_on_the_medium_workload():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "medium", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["config"]["workload"].startswith("medium") and d["steps"] == 2 and d["value"] > 0


def test_issue_roofline_of_the_shadow_kernel():
    sys.path.insert(0, ROOT)
    import bench
    # the city's update: 23.9G shadow rays in 1.344 s on 152 SMs at 2070 MHz
    r = bench.issue_roofline("large", "shadow", 23.9e9, 1.344, 152, 2070.0)
    per_ray = bench.NCU_SHADOW_INST["large"][0] / bench.NCU_SHADOW_INST["large"][1]
    assert abs(r["achieved"] - per_ray * 23.9e9 / 1.344 / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 4 * 2070e6 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12 and 0.0 < r["frac"] < 1.0
    assert bench.issue_roofline("large", "paths", 23.9e9, 1.344, 152, 2070.0) is None
    assert bench.issue_roofline("paper", "shadow", 2.1e4, 1e-4, 152, 2070.0) is None
    assert bench.issue_roofline("large", "shadow", 23.9e9, 1.344, 152, None) is None
