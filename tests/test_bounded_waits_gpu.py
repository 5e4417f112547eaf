"""Failure detection of the D3Q19 bulk kernel without a GPU fault.

The kernel waits for the bulk tensor copies of each plane stage on an mbarrier
with a time limit.  A test hook (lbm_debug_withhold_copy) makes one block of the
launch skip the copies of one stage, so that its wait runs out: the block must
record LBM_ERR_TIMEOUT, wait for the copies it did issue and return, the other
blocks must finish, and the device context must stay usable (a fresh run after
it is bitwise equal to a run in a fresh handle).
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402

# one periodic D3Q19 level of 96 x 32 x 16 nodes: column (1, 1) of the 32 x 8 tiling
# (x in [32, 64), y in [8, 16)) is staged by bulk tensor copies (it meets no seam)
DESC = {"lattice": 19, "coarse_n": (96, 32, 16), "boxes": [], "nu0": 1e-5, "storage": "f32",
        "init": {"kind": "vortex", "xc": 47.3, "yc": 15.6, "Rc": 4.0, "swirl": 0.05, "U": (0.05, 0.01, 0.0)}}


def _init(g):
    r, u = W.init_fields(DESC, 0)
    g.init_fields(0, r, u)


@pytest.mark.parametrize("use_graphs", [False, True])
def test_withheld_stage_copy_times_out_and_context_survives(use_graphs):
    g = lbm.Hierarchy(DESC, use_graphs=use_graphs)
    _init(g)
    g.advance(1)
    g.check_status()
    g.debug_withhold_copy(0, (1, 1, 0), 2, 200_000)  # 200 ms limit
    t0 = time.perf_counter()
    g.advance(1)
    rc = lbm.lib().lbm_check_status(g._h)
    dt = time.perf_counter() - t0
    assert rc == lbm.LBM_ERR_TIMEOUT, rc
    assert dt < 30.0
    # the hook off, the same handle and a fresh one give the same bits again
    g.debug_withhold_copy(-1, (0, 0, 0), 0, 1)
    _init(g)
    g.advance(3)
    g.check_status()
    h = lbm.Hierarchy(DESC, use_graphs=use_graphs)
    _init(h)
    h.advance(3)
    h.check_status()
    assert np.array_equal(g.get_pops(0), h.get_pops(0))


def test_withhold_hook_rejects_bad_arguments():
    g = lbm.Hierarchy(DESC)
    with pytest.raises(lbm.LbmError):
        g.debug_withhold_copy(0, (9, 0, 0), 0, 1000)
    with pytest.raises(lbm.LbmError):
        g.debug_withhold_copy(0, (1, 1, 0), 0, 0)
    d2 = {"lattice": 9, "coarse_n": (32, 32), "boxes": [], "nu0": 1e-5}
    with pytest.raises(lbm.LbmError):
        lbm.Hierarchy(d2).debug_withhold_copy(0, (0, 0, 0), 0, 1000)
