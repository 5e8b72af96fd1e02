"""The reference arm of bench.py (the oracle timed on the host cores) runs on
the CPU alone and never loads the CUDA library: its process maps the oracle's
shared object and not libpes.so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import contextlib, io, json, sys
sys.path.insert(0, {root!r})
import bench
args = bench.parse_args(["--impl", "reference", "--workload", "p1", "--d", "8", "--k", "2",
                         "--steps", "1", "--warmup", "0", "--cpu-sample-vars", "3"])
buf = io.StringIO()
with contextlib.redirect_stdout(buf):
    rc = bench.reference_arm(args, 1, 0)
maps = open("/proc/self/maps").read()
print(json.dumps({{"rc": rc, "line": buf.getvalue().strip().splitlines()[-1],
                  "libpes": "libpes" in maps, "liboracle": "liboracle" in maps}}))
"""


def test_reference_arm_loads_only_the_oracle():
    out = subprocess.run([sys.executable, "-c", PROBE.format(root=ROOT)], capture_output=True, text=True,
                         check=True, cwd=ROOT)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["rc"] == 0
    assert res["liboracle"] and not res["libpes"]
    line = json.loads(res["line"])
    assert line["impl"] == "reference" and line["value"] > 0
    conv = line["cpu_baseline"]["convolutions_per_step"]
    assert conv == {"credited_reverse_mode": 6, "executed_by_oracle": 9}
