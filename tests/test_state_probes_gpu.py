"""Checkpoint/resume, density probes and the stream-ordered level reduction through
the C-ABI."""
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


def _oracle_probe(o, x, y):
    """Bilinear density over the cell of the finest oracle level that holds (x, y)."""
    for l in reversed(range(o.n_levels)):
        lv = o.levels[l]
        n, off, per = lv["n"], lv["off"], lv["periodic"]
        qx, qy = x * 2 ** l - off[0], y * 2 ** l - off[1]
        bx, by = int(math.floor(qx)), int(math.floor(qy))
        cells = [(bx, by), (bx + 1, by), (bx, by + 1), (bx + 1, by + 1)]
        cls = o.node_class(l).reshape(n[1], n[0])
        ok = True
        for cx, cy in cells:
            if not per[0] and not 0 <= cx < n[0]:
                ok = False
            if not per[1] and not 0 <= cy < n[1]:
                ok = False
            if ok and cls[cy % n[1], cx % n[0]] == O.HOLE:
                ok = False
        if not ok:
            continue
        rho = o.macros(l)[0].reshape(n[1], n[0])
        fx, fy = qx - bx, qy - by
        ws = [(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy]
        return sum(w * rho[cy % n[1], cx % n[0]] for w, (cx, cy) in zip(ws, cells))
    raise AssertionError("no level holds the point")


def test_probes_sample_interpolated_density():
    """A ring of 36 probes (Sec. 4.2 uses 36 pressure probes on a circle), sampled
    every coarse step, equals the bilinear interpolation of the oracle's density on
    the finest level holding each point (the ring crosses levels 1 and 2)."""
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0)
    g = _make(d)
    o = O.Hierarchy(d)
    for l in range(o.n_levels):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    xc, yc = d["init"]["xc"], d["init"]["yc"]
    ang = np.arange(36) * 2 * math.pi / 36
    pts = np.stack([xc + 9.3 * np.cos(ang), yc + 9.3 * np.sin(ang), 0 * ang], 1)
    g.set_probes(pts, capacity=30)
    g.advance(22)
    o.advance(22)
    got = g.get_probes()
    assert got.shape == (22, 36)
    want = np.array([_oracle_probe(o, x, y) for x, y in pts[:, :2]])
    assert np.max(np.abs(got[-1] - want)) < 1e-12
    assert np.max(np.abs(got[-1] - 1.0)) > 1e-7  # the pulse has reached the ring


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_async_reduce_equals_reduce_every_step(storage):
    """lbm_reduce_async enqueued after every coarse step into rows of a pinned host
    array (and into a CUDA tensor) gives, after one synchronisation, exactly the sums
    that lbm_reduce returns step by step on a twin hierarchy."""
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0, storage=storage)
    a, b = _make(d), _make(d)
    K, L = 6, 2
    rows = torch.zeros((K, 4), dtype=torch.float64).pin_memory()
    dev = torch.zeros((K, 4), dtype=torch.float64, device="cuda")
    want = []
    for k in range(K):
        a.advance(1)
        a.reduce_async(L, rows[k])
        a.reduce_async(0, dev[k])
        b.advance(1)
        want.append((b.reduce(L), b.reduce(0)))
    a.synchronize()
    torch.cuda.synchronize()
    for k in range(K):
        assert np.array_equal(rows[k].numpy(), want[k][0])
        assert np.array_equal(dev[k].cpu().numpy(), want[k][1])
    # a numpy view of pinned memory is accepted too
    view = torch.zeros(4, dtype=torch.float64).pin_memory().numpy()
    a.reduce_async(1, view)
    a.synchronize()
    assert np.array_equal(view, a.reduce(1))
    a.check_status()


def test_async_reduce_rejects_pageable_host_memory():
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0, storage="f32")
    h = _make(d)
    with pytest.raises(lbm.LbmError) as e:
        h.reduce_async(0, np.zeros(4))
    assert e.value.code == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError):
        h.reduce_async(h.n_levels, torch.zeros(4, dtype=torch.float64).pin_memory())
