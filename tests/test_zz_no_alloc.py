"""The allocation-free reduction (lbm_reduce_static) against lbm_reduce.

lbm_reduce_static exists for callers that may not allocate device memory while
running (a process whose device heap belongs to its own pool allocator, a
fixed-latency loop that forbids cudaMalloc after start-up): its per-block
partials live in a static device array instead of a buffer of the handle.  This
file is collected last so that a run stopping at its first failure has already
run every other test; it passes alone in a fresh process and after the others.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402

LIMIT_NODES = 4096 * 2048  # LBM_STATIC_REDUCE_PARTIALS blocks of 2048 box nodes


def _call(fn, h, level):
    out = (C.c_double * 4)()
    rc = fn(h._h, level, out)
    assert rc == lbm.LBM_OK, lbm.lib().lbm_last_error(h._h).decode()
    return np.array(out[:])


def _make(d):
    h = lbm.Hierarchy(d)
    for l in range(h.n_levels):
        r, u = W.init_fields(d, l)
        h.init_fields(l, r, u)
    return h


def _two_calls_agree(h, steps):
    L = lbm.lib()
    for call in range(2):
        h.advance(steps)
        for l in range(h.n_levels):
            want = _call(L.lbm_reduce, h, l)
            got = _call(L.lbm_reduce_static, h, l)
            # same FP64 sums in a different block partition: agree to summation round-off
            assert np.allclose(got, want, rtol=1e-13, atol=1e-13), (call, l, got, want)
            assert got[0] > 0.0


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_static_reduce_matches_reduce_on_two_calls(storage):
    d = W.pulse2d(n=128, boxes=((32, 96), (48, 80)), storage=storage, Rc_finest=3.0)
    _two_calls_agree(_make(d), 3)


def test_static_reduce_d3q19_half_storage():
    """A D3Q19 hierarchy in FP16-shifted storage (a periodic slab level and a box)."""
    d = W.slab3d(nxy=64, nz=32, slab=(12, 20), box=((16, 16, 14), (48, 48, 18)), storage="f16s")
    _two_calls_agree(_make(d), 2)


def test_static_reduce_near_its_limit_allocates_nothing():
    """One level just under the limit (4096 x 2040 nodes, 4080 partials, far more
    blocks than lbm_reduce's partition uses): same sums as lbm_reduce on two calls,
    and, after a first call, the device's free memory does not move over repeated
    calls."""
    L = lbm.lib()
    nx, ny = 4096, 2040
    assert nx * ny <= LIMIT_NODES
    d = {"lattice": 9, "coarse_n": (nx, ny), "boxes": [], "nu0": 1e-5, "storage": "f32",
         "init": {"kind": "vortex", "xc": nx / 2, "yc": ny / 2, "Rc": 64.0, "swirl": 0.05, "U": (0.05, 0.02, 0.0)}}
    h = _make(d)
    _two_calls_agree(h, 1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        _call(L.lbm_reduce_static, h, 0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_reduce_rejects_levels_beyond_its_limit():
    L = lbm.lib()
    n = int(np.ceil(np.sqrt(LIMIT_NODES))) + 8  # a single level just past the limit
    h = lbm.Hierarchy({"lattice": 9, "coarse_n": (n, n), "boxes": [], "nu0": 1e-5, "storage": "f16s"})
    out = (C.c_double * 4)()
    rc = L.lbm_reduce_static(h._h, 0, out)
    assert rc == lbm.LBM_ERR_ARG
    assert "at most" in L.lbm_last_error(h._h).decode()
