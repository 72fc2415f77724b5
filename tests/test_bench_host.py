"""Host-side checks of bench.py: the reference arm's JSON line, the per-step
launch count and the DRAM-traffic records (no GPU needed)."""
import json
import os
import subprocess
import sys

import bench
import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Args:
    workload, tau, kT_fluid, streaming, box = "translocation", 1.0, 0.0, "pull", 256


def test_launches_per_step():
    p = bench.workload(0, "f32", _Args())
    # gather, MD cycle, stream-collide, spread sum (two kernels) and apply
    assert bench.launches_per_step(p) == 6
    # 16-bit storage: the apply converts the sums (one sum kernel)
    for st in ("f16", "bf16"):
        assert bench.launches_per_step(bench.workload(0, st, _Args())) == 5
    # a small box: the MD branch sets the step, the apply converts the sums
    a = _Args()
    a.workload = "small"
    assert bench.launches_per_step(bench.workload(0, "f32", a)) == 5
    a = _Args()
    a.workload = "solvent"
    assert bench.launches_per_step(bench.workload(0, "f32", a)) == 1
    a.kT_fluid = 1e-5
    assert bench.launches_per_step(bench.workload(0, "f32", a)) == 2


def test_traffic_records_name_the_bench_workload():
    with open(os.path.join(ROOT, "profiles", "lb_stream_collide_traffic.json")) as f:
        records = json.load(f)["records"]
    for r in records:
        assert r["kernel"] in bench.KERNEL_SOURCES
        assert r["storage"] in ("f32", "f16", "bf16")
        assert r["workload"] == bench.workload_name(bench.workload(0, r["storage"], _Args()))
        assert len(r["kernel_rev"]) == 16 and r["bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(ROOT, r["source"]))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "coupled D3Q19 MLUPS"
    assert line["value"] > 0 and line["unit"] == "MLUPS" and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("translocation 256x128x128")
