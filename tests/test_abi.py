"""The C-ABI library loads and exports every entry point include/lbm.h declares,
and host-side validation rejects malformed descriptions before any device work
(no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2004_14887_gb300 import build as B
from paper_2004_14887_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return lbm.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(lbm_\w+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)
    # the binding knows every declared entry point
    assert set(names) <= set(lbm.EXPORTS)


def test_library_is_built_for_sm_103a(L):
    """The build targets sm_103a only, with no PTX for other architectures."""
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_desc_struct_layout_matches_header(L):
    """Field offsets of the ctypes mirror follow the C declaration order and alignment."""
    d = lbm.lbm_hierarchy_desc
    assert d.coarse_n.offset == 8
    assert d.box_lo.offset == 32
    assert d.box_hi.offset == 32 + 96
    assert d.nu0.offset == 32 + 192
    assert d.alloc.offset % 8 == 0
    assert d.u_shift.offset == d.alloc_ctx.offset + 8
    assert C.sizeof(d) == d.u_shift.offset + 24


@pytest.mark.parametrize("bad,match", [
    ({"lattice": 7}, "lattice"),
    ({"boxes": [((30, 30), (40, 40))]}, "margin|seam"),
    ({"boxes": [((10, 10), (11, 11))]}, "4 parent cells"),
    ({"boxes": [((8, 8), (24, 24)), ((9, 9), (20, 20))]}, "margin"),
    ({"nu0": -1.0}, "nu0"),
    ({"dc_variant": 3}, "dc_variant"),
    ({"storage": "f16s", "u_shift": (0.5, 0.0, 0.0)}, "u_shift"),
    ({"storage": "f16s", "u_shift": (0.05, 0.0, 0.01)}, "u_shift"),
])
def test_malformed_descriptions_are_rejected_on_the_host(L, bad, match):
    desc = {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": 1e-5}
    desc.update(bad)
    d = lbm.make_desc(desc)
    h = C.c_void_p()
    rc = L.lbm_create_hierarchy(C.byref(d), None, C.byref(h))
    assert rc == lbm.LBM_ERR_BAD_DESC
    assert not h.value
    assert re.search(match, L.lbm_create_error().decode())


def test_binding_refuses_without_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA device"):
        lbm.Hierarchy({"lattice": 9, "coarse_n": (32, 32), "boxes": [], "nu0": 1e-5})


@pytest.mark.parametrize("desc", [
    {"lattice": 9, "coarse_n": (72, 40), "boxes": [], "nu0": 1e-5},
    {"lattice": 9, "coarse_n": (128, 128), "boxes": [((32, 32), (96, 96))], "nu0": 1e-5},
    {"lattice": 9, "coarse_n": (512, 512), "boxes": [((128, 128), (384, 384)), ((192, 192), (320, 320))], "nu0": 1e-5},
    {"lattice": 9, "coarse_n": (64, 64), "boxes": [((16, 0), (48, 64))], "nu0": 1e-5},
    {"lattice": 19, "coarse_n": (16, 16, 24), "boxes": [((0, 0, 6), (16, 16, 18)), ((4, 4, 9), (12, 12, 15))],
     "nu0": 1e-5},
    {"lattice": 19, "coarse_n": (32, 32, 32), "boxes": [((8, 8, 8), (24, 24, 24)), ((12, 12, 12), (20, 20, 20))],
     "nu0": 1e-5},
], ids=["2d-periodic-ragged", "2d-2lvl", "2d-3lvl-512", "2d-slab", "3d-slab-3lvl", "3d-cubes-3lvl"])
def test_host_geometry_and_tile_rule_accept_valid_hierarchies(L, desc):
    """Host-side set-up (classes, interface tables, and the check that the kernels'
    geometric tile rule matches the node-by-node classification of every tile) runs
    before any device work; without a GPU the call then stops at the first CUDA call."""
    d = lbm.make_desc(desc)
    h = C.c_void_p()
    rc = L.lbm_create_hierarchy(C.byref(d), None, C.byref(h))
    if rc == lbm.LBM_OK:
        L.lbm_destroy(h)
    else:
        assert rc == lbm.LBM_ERR_CUDA, L.lbm_create_error().decode()


def test_batch_validation_on_the_host(L):
    """Batches take D2Q9 members with one storage and level count."""
    from paper_2004_14887_gb300 import workloads as W

    descs = W.batch2d(n=3, sides=(48, 64))
    arr = (lbm.lbm_hierarchy_desc * 3)(*[lbm.make_desc(d) for d in descs])
    arr[1].storage = 0 if arr[0].storage else 1
    h = C.c_void_p()
    assert L.lbm_create_batch(arr, 3, None, C.byref(h)) == lbm.LBM_ERR_BAD_DESC
    arr[1].storage = arr[0].storage
    arr[2].lattice = 19
    assert L.lbm_create_batch(arr, 3, None, C.byref(h)) == lbm.LBM_ERR_BAD_DESC
    assert L.lbm_create_batch(arr, 0, None, C.byref(h)) == lbm.LBM_ERR_ARG


def _create_masked(L, desc, masks):
    d = lbm.make_desc(desc)
    keep = [None if m is None else np.ascontiguousarray(np.asarray(m, np.uint8)) for m in masks]
    arr = (C.c_void_p * lbm.MAX_LEVELS)()
    for l, m in enumerate(keep):
        if l > 0 and m is not None:
            arr[l] = m.ctypes.data
    h = C.c_void_p()
    rc = L.lbm_create_hierarchy_masked(C.byref(d), arr, None, C.byref(h))
    if rc == lbm.LBM_OK:
        L.lbm_destroy(h)
    return rc


def test_staircase_hierarchies_pass_the_host_set_up(L):
    """Circular and inclined staircase regions and an L-shaped one: classes, interface
    tables and per-tile classes are built on the host (no GPU: the call stops at the
    first CUDA call)."""
    from paper_2004_14887_gb300 import workloads as W

    for d in (W.pulse_circle(), W.vortex_inclined()):
        rc = _create_masked(L, d, d["masks"])
        assert rc in (lbm.LBM_OK, lbm.LBM_ERR_CUDA), L.lbm_create_error().decode()


@pytest.mark.parametrize("case,match", [
    ("diagonal", "corner only"),
    ("not_finest", "finest level"),
    ("d3q19", "2-D only"),
    ("spanning", "spans no axis"),
])
def test_invalid_staircase_masks_are_rejected(L, case, match):
    desc = {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": 1e-5}
    m = np.ones((16, 16), np.uint8)
    masks = [None, m]
    if case == "diagonal":
        m[8:, 8:] = 0
        m[:8, :8] = 0  # the two refined quadrants meet at (16, 16) only
    elif case == "not_finest":
        desc["boxes"] = [((8, 8), (24, 24)), ((12, 12), (20, 20))]
        masks = [None, m, None]
    elif case == "d3q19":
        desc = {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5}
        masks = [None, np.ones((8, 8, 8), np.uint8)]
    elif case == "spanning":
        desc["boxes"] = [((8, 0), (24, 32))]
        masks = [None, np.ones((32, 16), np.uint8)]
    assert _create_masked(L, desc, masks) == lbm.LBM_ERR_BAD_DESC
    assert re.search(match, L.lbm_create_error().decode())
