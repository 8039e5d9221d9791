"""Host-side pieces of bench.py (no GPU): the workload descriptions both arms print, and the
reference arm (the CPU oracle on a bounded slab) for every workload, at small sizes."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("wl", ["nsf", "mhd", "adr", "nsf12", "mhd18", "hcnsf"])
def test_workload_descriptions(wl):
    case = bench.make_case(wl, 16)
    K, q = bench.kq(wl)
    cfg = bench.config_of(wl, case, "fp32", K, q)
    dim = 3 if wl in bench.DIM3 else 2
    assert cfg["grid"] == [16] * dim and cfg["components"] == K and cfg["velocities"] == q
    assert cfg["workload"] == f"{wl}_{bench.LATTICE_NAME[wl]}_{'x'.join(['16'] * dim)}_fp32"
    assert bench.cells(wl, case) == 16 ** dim
    Q = bench.fields(wl, case)
    assert tuple(Q.shape) == (K,) + (16,) * dim


@pytest.mark.parametrize("wl", ["nsf", "hcnsf"])
def test_reference_arm_prints_one_json_line(wl):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", wl,
                        "--n", "16", "--steps", "2", "--warmup", "3"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "LUP/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith(wl + "_")
