"""The op-counting build of the oracle (oracle/opcount/count_flops.py) still
applies to the oracle's source, compiles, and counts plausible per-cell flops
on a small magnetosphere grid (the algorithmic figures of the roofline come
from it)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_op_counting_build_counts_the_sweeps():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "oracle", "opcount", "count_flops.py"), "32", "24", "24"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = {l.split(" {")[0]: ast.literal_eval("{" + l.split(" {", 1)[1]) for l in r.stdout.splitlines() if " {" in l}
    assert 150 < lines["cfl"]["flops"] < 260
    for axis in "xyz":
        c = lines[f"sweep {axis}"]
        assert 1000 < c["flops"] < 2500, c
        assert c["div"] > 50 and c["sqrt"] > 5
