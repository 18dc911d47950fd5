"""bench.py's reference arm (the oracle on the host cores) prints the one JSON
line of the benchmark contract, on a small grid (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--grid", "32", "24", "24"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "cell-updates/s per full xyz step"
    assert d["unit"] == "cell-updates/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("magnetosphere_32x24x24")


def test_traffic_table_is_keyed_to_code_not_comments():
    """The ncu traffic entries are keyed to a hash of the kernels' code: a
    comment edit keeps them, a code edit marks them stale; every entry names
    a kernel whose sources are listed."""
    sys.path.insert(0, ROOT)
    import bench
    base = "int f(int a) { return a + 1; }\n"
    assert bench._code_only(base) == bench._code_only("// one\n" + base + "/* two\n three */\n\n")
    assert bench._code_only(base) != bench._code_only(base.replace("+ 1", "+ 2"))
    for key, entry in bench.NCU_TRAFFIC.items():
        prec, kern = key.split(":")
        assert f"{prec}:{'cfl' if kern == 'cfl' else 'sweep'}" in bench.KERNEL_SOURCES
        assert entry["bytes_per_cell"] > 0 and len(entry["src"]) == 16
    assert len(bench.kernel_source_hash("fp64:x")) == 16
