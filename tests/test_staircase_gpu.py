"""Staircase refinement interfaces of arbitrary shape on the GPU (paper Sec. 4.1.2
circular interface, Sec. 4.2.2 inclined interface, App. B corners) against the FP64
oracle, through the C-ABI (lbm_create_hierarchy_masked).

* node classes equal the oracle's on circular, inclined and L-shaped regions;
* FP64 runs match the oracle to 1e-12 (relative L-infinity, and relative to the signal);
* a mask that refines the whole box runs bit for bit like the box;
* every tile shape of the 2-D bulk kernel (per-tile classes for staircase levels) gives
  the same bits;
* the dual-cell weights of a staircase hierarchy tile the domain (total mass of a
  density-1 state = domain area);
* FP32 storage stays within the precision bound derived in test_signal_parity_gpu.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402


def _l_shape(steps=40):
    d = W.vortex2d(n=32, patch=(8, 24), steps=steps, Rc=3.0, centre=(14.0, 14.0))
    m = np.ones((16, 16), np.uint8)
    m[8:, 8:] = 0
    d["masks"] = [None, m]
    d["name"] = "vortex_l_shape_32"
    return d


CASES = {
    # the pulse in a Mach-0.1 mean flow: the relative L-infinity of u is then taken
    # against a velocity of the lattice's scale, as in the box cases
    "circle": lambda: W.pulse_circle(steps=60, mach=0.1),
    "inclined": lambda: W.vortex_inclined(steps=60),
    "L": _l_shape,
}


def _pair(d, threaded=True):
    g = lbm.Hierarchy(d)
    o = O.Hierarchy(d, threaded=threaded)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
        o.init(l, r, u)
    return g, o


@pytest.mark.parametrize("case", list(CASES))
def test_staircase_classes_match_oracle(case):
    d = CASES[case]()
    g = lbm.Hierarchy(d)
    o = O.Hierarchy(d)
    for l in range(g.n_levels):
        assert g.levels[l]["n"] == o.levels[l]["n"]
        assert np.array_equal(g.node_class(l), o.node_class(l))


@pytest.mark.parametrize("case", list(CASES))
def test_staircase_f64_matches_oracle(case):
    d = CASES[case]()
    g, o = _pair(d)
    g.advance(d["steps"])
    o.advance(d["steps"])
    g.check_status()
    amp = max(float(np.max(np.abs(o.macros(l)[0][o.node_class(l) != O.HOLE] - 1.0))) for l in range(2))
    for l in range(g.n_levels):
        m = g.node_class(l) != lbm.HOLE
        rg, ug = g.get_macros(l)
        ro, uo = o.macros(l)
        er = np.max(np.abs(rg[m] - ro[m])) / np.max(np.abs(ro[m]))
        eu = np.max(np.abs(ug[:, m] - uo[:, m])) / np.max(np.abs(uo[:, m]))
        ed = np.max(np.abs(rg[m] - ro[m])) / amp
        assert er <= 1e-12 and eu <= 1e-12 and ed <= 1e-9, (case, l, er, eu, ed)
    assert 1 <= g.max_newton_iters() <= 3


def test_full_mask_runs_like_the_box():
    d = W.vortex2d(n=32, patch=(8, 24), steps=10)
    dm = dict(d, masks=[None, np.ones((16, 16), np.uint8)])
    a, _ = _pair(d)
    b, _ = _pair(dm)
    a.advance(10)
    b.advance(10)
    for l in range(2):
        assert np.array_equal(a.get_pops(l), b.get_pops(l))


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_every_tile_shape_on_a_staircase_gives_the_same_bits(storage):
    d = dict(W.vortex_inclined(steps=8), storage=storage)
    ref, _ = _pair(d)
    ref.advance(8)
    for c in range(lbm.TILE_CONFIGS):
        g, _ = _pair(d)
        for l in range(g.n_levels):
            g.set_tile_config(l, c)
        g.advance(8)
        for l in range(g.n_levels):
            assert np.array_equal(g.get_pops(l), ref.get_pops(l)), (c, l)


@pytest.mark.parametrize("case", ["circle", "inclined", "L"])
def test_staircase_weights_tile_the_domain(case):
    d = CASES[case]()
    d["init"] = {"kind": "uniform", "rho": 1.0, "U": (0.0, 0.0, 0.0)}
    g = lbm.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
    total = sum(g.reduce(l)[0] for l in range(g.n_levels))
    n = d["coarse_n"][0] * d["coarse_n"][1]
    assert abs(total - n) < 1e-9 * n


def test_staircase_f32_within_the_derived_bound():
    from tests.test_signal_parity_gpu import derived_bounds

    d64 = W.pulse_circle(steps=40)
    o = O.Hierarchy(d64, threaded=True)
    for l in range(2):
        r, u = W.init_fields(d64, l)
        o.init(l, r, u)
    o.advance(40)
    d = dict(d64, storage="f32")
    g = lbm.Hierarchy(d)
    for l in range(2):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
    g.advance(40)
    br, bu = derived_bounds(d, o, 40)
    for l in range(2):
        m = g.node_class(l) != lbm.HOLE
        rg, ug = g.get_macros(l)
        ro, uo = o.macros(l)
        assert np.max(np.abs(rg[m] - ro[m])) <= br
        assert np.max(np.abs(ug[:, m] - uo[:, m])) <= bu


def test_probes_are_refused_on_a_staircase_hierarchy():
    g = lbm.Hierarchy(W.pulse_circle())
    with pytest.raises(lbm.LbmError) as e:
        g.set_probes(np.array([[32.0, 32.0, 0.0]]), 4)
    assert e.value.code == lbm.LBM_ERR_ARG
