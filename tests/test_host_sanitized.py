"""The library's host code under the undefined-behaviour sanitizer: the CUDA library
is rebuilt with its host code instrumented (-fsanitize=undefined, no recovery) into a
private directory, and the host-side set-up of several hierarchies (geometry, node
classes, interface sets and stencils, the check of the kernels' geometric tile and
plane rules) runs in a subprocess until the first device call, which fails cleanly
without a GPU.  The first undefined operation aborts the subprocess."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, ctypes as C
sys.path.insert(0, {root!r})
from paper_2004_14887_gb300 import lbm
lbm.LIB_PATH = {lib!r}
L = lbm.lib()
descs = [
    {{"lattice": 9, "coarse_n": (72, 40), "boxes": [], "nu0": 1e-5}},
    {{"lattice": 9, "coarse_n": (512, 512), "boxes": [((128, 128), (384, 384)), ((192, 192), (320, 320))],
      "nu0": 1e-5}},
    {{"lattice": 9, "coarse_n": (64, 64), "boxes": [((16, 0), (48, 64))], "nu0": 1e-5, "dc_variant": 1}},
    {{"lattice": 19, "coarse_n": (16, 16, 24), "boxes": [((0, 0, 6), (16, 16, 18)), ((4, 4, 9), (12, 12, 15))],
      "nu0": 1e-5}},
    {{"lattice": 19, "coarse_n": (34, 20, 16), "boxes": [((8, 4, 4), (24, 16, 12))], "nu0": 1e-5,
      "storage": "f16s", "u_shift": (0.05, 0.01, 0.0)}},
]
for desc in descs:
    d = lbm.make_desc(desc)
    h = C.c_void_p()
    rc = L.lbm_create_hierarchy(C.byref(d), None, C.byref(h))
    if rc == lbm.LBM_OK:
        L.lbm_destroy(h)
    elif rc != lbm.LBM_ERR_CUDA:
        raise SystemExit("rc %d: %s" % (rc, L.lbm_create_error().decode()))
print("clean")
"""


@pytest.mark.slow
@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc is required")
def test_host_setup_has_no_undefined_behaviour(tmp_path):
    src = os.path.join(ROOT, "paper_2004_14887_gb300", "csrc", "lbm_host.cu")
    lib = str(tmp_path / "liblbm_ubsan.so")
    try:
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
                        "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-Xcompiler", "-fsanitize=undefined",
                        "-Xcompiler", "-fno-sanitize-recover=all", "-I", os.path.join(ROOT, "include"), "-shared",
                        "-o", lib, src, "-lcudart", "-lubsan"], check=True, capture_output=True, text=True,
                       timeout=900)
    except subprocess.CalledProcessError as e:  # pragma: no cover - toolchain without the runtime
        pytest.skip(f"no UBSan build: {e.stderr[-200:]}")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, lib=lib)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, (r.stdout[-500:], r.stderr[-2000:])
    assert "runtime error" not in r.stderr, r.stderr[-2000:]
