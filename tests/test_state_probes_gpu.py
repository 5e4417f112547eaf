"""Checkpoint/resume and density probes through the C-ABI."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402


def _make(d):
    h = lbm.Hierarchy(d)
    for l in range(h.n_levels):
        r, u = W.init_fields(d, l)
        h.init_fields(l, r, u)
    return h


@pytest.mark.parametrize("storage", ["f64", "f16s"])
def test_save_load_resumes_bit_for_bit(storage):
    """2n steps in one run equal n steps, save, load into a fresh handle, n steps."""
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0, storage=storage)
    a = _make(d)
    a.advance(7)
    buf = a.save_state()
    a.advance(7)
    b = lbm.Hierarchy(d)
    b.load_state(buf)
    b.advance(7)
    for l in range(a.n_levels):
        assert np.array_equal(a.get_pops(l), b.get_pops(l))


def test_load_rejects_foreign_state():
    a = _make(W.vortex2d(n=32, patch=(8, 24)))
    b = lbm.Hierarchy(W.vortex2d(n=48, patch=(12, 36)))
    with pytest.raises(lbm.LbmError):
        b.load_state(a.save_state())


def test_probes_sample_interpolated_density():
    """A ring of 36 probes (Sec. 4.2 uses 36 pressure probes on a circle), sampled
    every coarse step, equals the bilinear interpolation of the oracle's density."""
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0)
    g = _make(d)
    o = O.Hierarchy(d)
    for l in range(o.n_levels):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    ang = np.arange(36) * 2 * math.pi / 36
    pts = np.stack([32 + 24 * np.cos(ang), 32 + 24 * np.sin(ang), 0 * ang], 1)
    g.set_probes(pts, capacity=10)
    g.advance(6)
    o.advance(6)
    got = g.get_probes()
    assert got.shape == (6, 36)
    # level 0 holds every ring point (radius 24 > the level-1 patch half-width 16)
    rho, _ = o.macros(0)
    rho = rho.reshape(64, 64)
    x, y = pts[:, 0], pts[:, 1]
    x0, y0 = np.floor(x).astype(int), np.floor(y).astype(int)
    fx, fy = x - x0, y - y0
    want = (rho[y0, x0] * (1 - fx) * (1 - fy) + rho[y0, (x0 + 1) % 64] * fx * (1 - fy)
            + rho[(y0 + 1) % 64, x0] * (1 - fx) * fy + rho[(y0 + 1) % 64, (x0 + 1) % 64] * fx * fy)
    assert np.max(np.abs(got[-1] - want)) < 1e-12
    assert np.max(np.abs(got[-1] - 1.0)) > 1e-7  # the pulse has reached the ring
