"""Host logic of the benchmark: the reference arm (the oracle on the host
cores) prints a JSON line with the GPU arm's metric, unit and workload
configuration and the keys of the contract (cpu_baseline, e2e with zero
transfers); the revision that validates stored ncu traffic follows the
kernel's code, not its comments."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_matches_the_gpu_arm():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-rows", "8"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    want = bench.workload_config(bench.REF_FRAC_BITS, d["config"]["R"], 1, "not applicable (host cores)")
    assert d["config"] == want
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_revision_follows_code_not_comments(tmp_path, monkeypatch):
    # the stored ncu traffic stays valid across comment edits of the
    # kernel's sources and is dropped by any change of code
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    monkeypatch.setitem(bench.KERNEL_SOURCES, "probe", [str(src)])
    src.write_text("// sum\n__global__ void k(int* p) { p[0] += 1; /* one */ }\n")
    r0 = bench.kernel_revision("probe")
    src.write_text("// the sum, reworded\n__global__ void k(int* p) {\n  p[0] += 1;  /* still one */\n}\n")
    assert bench.kernel_revision("probe") == r0
    src.write_text("// sum\n__global__ void k(int* p) { p[0] += 2; /* one */ }\n")
    assert bench.kernel_revision("probe") != r0
