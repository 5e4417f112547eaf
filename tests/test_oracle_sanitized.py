"""The oracle under the undefined-behaviour sanitizer: the C oracle is rebuilt with
-fsanitize=undefined (no recovery: the first undefined operation aborts) into a
private directory and advances small 2- and 3-level D2Q9 and D3Q19 hierarchies in a
subprocess, so out-of-range shifts, signed overflow, misaligned or out-of-bounds
array indexing detected by UBSan fail the test.  Host-side check of the test
infrastructure; no GPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
from oracle import oracle as O
from paper_2004_14887_gb300 import workloads as W
O.LIB_PATH = {lib!r}
O.build = lambda force=False: O.LIB_PATH
cases = [
    W.vortex2d(n=32, patch=(8, 24)),
    W.pulse2d(n=48, boxes=((12, 36), (18, 30)), Rc_finest=3.0),
    {{"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5,
      "init": {{"kind": "vortex", "xc": 8.3, "yc": 7.6, "Rc": 2.0, "swirl": 0.05, "U": (0.05, 0.01, 0.02),
                "noise": 0.01, "seed": 1}}}},
]
for d in cases:
    o = O.Hierarchy(d)
    for l in range(o.n_levels):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    o.advance(3)
print("clean")
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc is required")
def test_oracle_has_no_undefined_behaviour(tmp_path):
    src = os.path.join(ROOT, "oracle", "dc_lbm_oracle.c")
    lib = str(tmp_path / "liblbm_oracle_ubsan.so")
    try:
        subprocess.run(["gcc", "-O1", "-g", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fsanitize=undefined", "-fno-sanitize-recover=all", "-o", lib, src, "-lm"],
                       check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:  # pragma: no cover - toolchain without the runtime
        pytest.skip(f"no UBSan runtime: {e.stderr[-200:]}")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, lib=lib)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-2000:]
    assert "runtime error" not in r.stderr, r.stderr[-2000:]
