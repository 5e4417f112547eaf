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


def _call(fn, h, level):
    out = (C.c_double * 4)()
    rc = fn(h._h, level, out)
    assert rc == lbm.LBM_OK, lbm.lib().lbm_last_error(h._h).decode()
    return np.array(out[:])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_static_reduce_matches_reduce_on_two_calls(storage):
    L = lbm.lib()
    d = W.pulse2d(n=128, boxes=((32, 96), (48, 80)), storage=storage, Rc_finest=3.0)
    h = lbm.Hierarchy(d)
    for l in range(h.n_levels):
        r, u = W.init_fields(d, l)
        h.init_fields(l, r, u)
    for call in range(2):
        h.advance(3)
        for l in range(h.n_levels):
            want = _call(L.lbm_reduce, h, l)
            got = _call(L.lbm_reduce_static, h, l)
            # same FP64 sums in a different block partition: agree to summation round-off
            assert np.allclose(got, want, rtol=1e-13, atol=1e-13), (call, l, got, want)
            assert got[0] > 0.0


def test_static_reduce_rejects_levels_beyond_its_limit():
    L = lbm.lib()
    limit = 4096 * 2048
    n = int(np.ceil(np.sqrt(limit))) + 8  # a single level just past the limit
    h = lbm.Hierarchy({"lattice": 9, "coarse_n": (n, n), "boxes": [], "nu0": 1e-5, "storage": "f16s"})
    out = (C.c_double * 4)()
    rc = L.lbm_reduce_static(h._h, 0, out)
    assert rc == lbm.LBM_ERR_ARG
    assert "at most" in L.lbm_last_error(h._h).decode()
