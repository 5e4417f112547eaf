"""GPU path (CUDA library through the C-ABI) against the FP64 CPU oracle, element
by element on the same seeded inputs.

Tolerances (relative L-infinity, max|gpu - oracle| / max|oracle| per field and
level over active nodes):
* FP64 storage: 1e-12 (the target the method's parity is stated at).
* FP32 storage, FP32 arithmetic: 5e-5 after 200 coarse steps.  Derivation: every
  update rounds each population to 2^-24 relative, ~2e-7 on the node's mass; at
  tau ~ 1/2 the off-equilibrium part flips sign every step and is damped only by
  the 2 % finite-difference share of the H-RR hybrid, so the errors random-walk
  over the n = 400 finest updates (x 20) and the maximum over ~3e4 nodes adds
  ~4.5 standard deviations: ~2e-5 on rho and on u (scale 0.1 absolute -> 1e-5
  relative x 2).  Measured: 4.6e-6 (rho), 1.8e-5 (u).
* FP16 shifted storage (f - w_i as IEEE half, FP32 arithmetic): the stored
  deviation |f - w_i| reaches ~0.1 w_i at Mach 0.1, quantised to 2^-11 of itself,
  i.e. ~5e-5 w_i per population and update; with the same growth this gives
  ~1e-3 absolute on rho-1 and u; the bound is 3e-3 relative on u.  Measured 2.1e-3.
"""
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

CS = 1.0 / math.sqrt(3.0)


def _pair(d, use_graphs=True):
    g = lbm.Hierarchy(d, use_graphs=use_graphs)
    o = O.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
        o.init(l, r, u)
    return g, o


def _rel_errors(g, o):
    """Per level: rel Linf of rho and u, and of rho against the largest density
    deviation |rho - 1| found on any level (the signal amplitude)."""
    rows, amp = [], 0.0
    for l in range(g.n_levels):
        m = g.node_class(l) != lbm.HOLE
        rg, ug = g.get_macros(l)
        ro, uo = o.macros(l)
        amp = max(amp, np.max(np.abs(ro[m] - 1.0)))
        rows.append((np.max(np.abs(rg[m] - ro[m])), np.max(np.abs(ro[m])),
                     np.max(np.abs(ug[:, m] - uo[:, m])), np.max(np.abs(uo[:, m]))))
    return [(dr / r, du / u, dr / max(amp, 1e-300)) for dr, r, du, u in rows]


def _assert_parity(g, o, tol, tol_dev=None):
    errs = _rel_errors(g, o)
    for l, (er, eu, edr) in enumerate(errs):
        assert er <= tol and eu <= tol, f"level {l}: rho {er:.3e} u {eu:.3e}"
        if tol_dev is not None:
            assert edr <= tol_dev, f"level {l}: rho-1 {edr:.3e}"
    return errs


@pytest.mark.parametrize("d", [
    {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": 1e-5},
    {"lattice": 9, "coarse_n": (48, 48), "boxes": [((12, 12), (36, 36)), ((18, 18), (30, 30))], "nu0": 1e-5},
    {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 0), (24, 32))], "nu0": 1e-5},
    {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5},
], ids=["2d-2lvl", "2d-3lvl", "2d-slab", "3d-2lvl"])
def test_node_classes_match_oracle(d):
    g = lbm.Hierarchy(d)
    o = O.Hierarchy(d)
    for l in range(g.n_levels):
        assert g.levels[l]["n"] == o.levels[l]["n"]
        assert g.levels[l]["off"] == o.levels[l]["off"]
        assert abs(g.levels[l]["tau"] - o.levels[l]["tau"]) < 1e-15
        assert np.array_equal(g.node_class(l), o.node_class(l))
        assert g.levels[l]["n_active"] == W.node_counts(d)[l]


def test_single_level_periodic_vortex_f64():
    d = {"lattice": 9, "coarse_n": (72, 40), "boxes": [], "nu0": 1e-5,
         "init": {"kind": "vortex", "xc": 30.3, "yc": 20.7, "Rc": 5.0, "swirl": 0.08, "U": (0.05, 0.02, 0.0)}}
    g, o = _pair(d)
    g.advance(25)
    o.advance(25)
    _assert_parity(g, o, 1e-12)


def test_vortex2d_two_level_full_workload_f64():
    """D2Q9, 128^2 with a 64^2-cell patch, vortex at Mach 0.1 crossing the
    interface, 200 coarse steps: GPU FP64 matches the oracle to 1e-12."""
    d = W.vortex2d()
    g, o = _pair(d)
    g.advance(d["steps"])
    o.advance(d["steps"])
    g.check_status()
    errs = _assert_parity(g, o, 1e-12, tol_dev=1e-9)
    print("vortex2d f64 rel Linf per level (rho, u, rho-1):", errs)
    assert 1 <= g.max_newton_iters() <= 3


def test_three_level_pulse_f64():
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), steps=30, Rc_finest=3.0)
    g, o = _pair(d)
    g.advance(30)
    o.advance(30)
    _assert_parity(g, o, 1e-12, tol_dev=1e-9)


def test_pulse2d_three_level_full_size_f64():
    """The 512^2 three-level workload at full size (1.65 M node updates per coarse
    step), 12 coarse steps, in the graph-replayed launch configuration of the bench."""
    d = W.pulse2d(steps=12)
    g, o = _pair(d)
    g.advance(12)
    o.advance(12)
    _assert_parity(g, o, 1e-12, tol_dev=1e-9)


def test_pulse2d_three_level_full_size_f32_bench_configuration():
    """The bench's default line: the same full-size workload in FP32 storage with the
    tile shapes the autotuner picks on the live state (as bench.py does), graph
    replayed, 12 coarse steps against the FP64 oracle (FP32 bound of this module)."""
    d = W.pulse2d(steps=12, storage="f32")
    g, o = _pair(d)
    g.autotune(reps=3)
    g.advance(12)
    o.advance(12)
    _assert_parity(g, o, 5e-5)


def test_dc1_variant_f64():
    d = W.vortex2d(n=64, patch=(16, 48), steps=40)
    d["dc_variant"] = 1
    g, o = _pair(d)
    g.advance(40)
    o.advance(40)
    _assert_parity(g, o, 1e-12)


def test_slab_level_periodic_axis_f64():
    d = W.vortex2d(n=64, patch=(16, 48), steps=30)
    d["boxes"] = [((16, 0), (48, 64))]
    g, o = _pair(d)
    g.advance(30)
    o.advance(30)
    _assert_parity(g, o, 1e-12)


def test_graph_replay_equals_eager_launches():
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), steps=14, Rc_finest=3.0)
    ga, _ = _pair(d, use_graphs=True)
    gb = lbm.Hierarchy(d, use_graphs=False)
    for l in range(gb.n_levels):
        r, u = W.init_fields(d, l)
        gb.init_fields(l, r, u)
    ga.advance(14)
    gb.advance(14)
    for l in range(ga.n_levels):
        assert np.array_equal(ga.get_pops(l), gb.get_pops(l))


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_uniform_flow_is_preserved(storage):
    d = {"lattice": 9, "coarse_n": (48, 48), "boxes": [((12, 12), (36, 36)), ((18, 18), (30, 30))], "nu0": 1e-5,
         "storage": storage, "init": {"kind": "uniform", "rho": 1.0, "U": (0.04, -0.03, 0.0)}}
    g = lbm.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
    g.advance(10)
    tol = {"f64": 1e-14, "f32": 5e-6, "f16s": 2e-3}[storage]
    for l in range(g.n_levels):
        m = g.node_class(l) != lbm.HOLE
        r, u = g.get_macros(l)
        assert np.max(np.abs(r[m] - 1.0)) < tol
        assert np.max(np.abs(u[0, m] - 0.04)) < tol and np.max(np.abs(u[1, m] + 0.03)) < tol


@pytest.mark.parametrize("storage,tol", [("f32", 5e-5), ("f16s", 3e-3)])
def test_reduced_precision_against_oracle(storage, tol):
    d = W.vortex2d(storage=storage)
    g, o = _pair(d)
    g.advance(d["steps"])
    o.advance(d["steps"])
    g.check_status()
    errs = _assert_parity(g, o, tol)
    print(f"vortex2d {storage} rel Linf per level (rho, u, rho-1):", errs)


def test_reduce_matches_weighted_oracle_sums():
    d = W.vortex2d(n=64, patch=(16, 48), steps=10)
    g, o = _pair(d)
    g.advance(10)
    o.advance(10)
    total = np.zeros(3)
    for l in range(g.n_levels):
        got = g.reduce(l)
        cls = o.node_class(l)
        f = o.pops(l)
        c, _ = O.lattice(9)
        n = o.levels[l]["n"]
        # dual-cell weights: outline nodes of the level keep the part of their cell inside it
        w = np.zeros(o.levels[l]["N"])
        for idx in range(len(w)):
            if cls[idx] == O.HOLE:
                continue
            x, y = idx % n[0], idx // n[0]
            own = 1.0
            if l == 1:
                own *= 0.5 if x in (0, n[0] - 1) else 1.0
                own *= 0.5 if y in (0, n[1] - 1) else 1.0
            child = 0.0
            if l == 0:
                cx = 0.5 if x in (16, 48) else (1.0 if 16 < x < 48 else 0.0)
                cy = 0.5 if y in (16, 48) else (1.0 if 16 < y < 48 else 0.0)
                child = cx * cy
            w[idx] = (own - child) / 4 ** l
        want = np.array([w @ f.sum(0), w @ (c[:, 0] @ f), w @ (c[:, 1] @ f)])
        assert np.allclose(got[:3], want, rtol=1e-13, atol=1e-12)
        total += got[:3]
    # the weights tile the domain: total mass ~ domain volume (density ~ 1)
    assert abs(total[0] / (64 * 64) - 1.0) < 1e-3


def test_nan_in_state_is_reported():
    d = {"lattice": 9, "coarse_n": (32, 32), "boxes": [], "nu0": 1e-5}
    g = lbm.Hierarchy(d)
    r = np.ones(32 * 32)
    r[100] = np.nan
    g.init_fields(0, r, np.zeros((2, 32 * 32)))
    with pytest.raises(lbm.LbmError) as e:
        g.reduce(0)
    assert e.value.code == lbm.LBM_ERR_DIVERGED


def test_device_tensors_in_and_out():
    d = W.vortex2d(n=32, patch=(8, 24))
    g, o = _pair(d)
    g.advance(3)
    o.advance(3)
    N = g.levels[1]["N"]
    rho = torch.empty(N, dtype=torch.float64, device="cuda")
    u = torch.empty((2, N), dtype=torch.float64, device="cuda")
    g.get_macros(1, out=(rho, u))
    torch.cuda.synchronize()
    ro, uo = o.macros(1)
    assert np.max(np.abs(rho.cpu().numpy() - ro)) < 1e-12
    assert np.max(np.abs(u.cpu().numpy() - uo)) < 1e-12


def test_d3q19_two_level_f64():
    d = {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5,
         "init": {"kind": "vortex", "xc": 9.3, "yc": 8.6, "Rc": 2.5, "swirl": 0.06, "U": (0.05, 0.01, 0.02),
                  "noise": 0.01, "seed": 3}}
    g, o = _pair(d)
    g.advance(6)
    o.advance(6)
    _assert_parity(g, o, 1e-12)


def test_d3q19_three_level_slab_f64():
    d = {"lattice": 19, "coarse_n": (16, 16, 24), "boxes": [((0, 0, 6), (16, 16, 18)), ((4, 4, 9), (12, 12, 15))],
         "nu0": 1e-5, "init": {"kind": "pulse+vortex", "xc": 8.2, "yc": 7.9, "zc": 12.1, "Rc": 1.5, "A": 1e-3,
                               "swirl": 0.05, "U": (0.05, 0.0, 0.0)}}
    g, o = _pair(d)
    g.advance(4)
    o.advance(4)
    _assert_parity(g, o, 1e-12)


def test_every_tile_shape_gives_identical_results(tmp_path):
    """The autotuner only changes the launch shape of the bulk kernel: every shape
    computes the same per-node arithmetic, so the state is bitwise identical; the
    tuned choice is cached and reloaded by (lattice, storage, level boxes)."""
    d = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), steps=8, Rc_finest=3.0, storage="f32")
    ref, _ = _pair(d)
    ref.advance(8)
    for c in range(lbm.TILE_CONFIGS):
        g, _ = _pair(d)
        for l in range(g.n_levels):
            g.set_tile_config(l, c)
        g.advance(8)
        for l in range(g.n_levels):
            assert np.array_equal(g.get_pops(l), ref.get_pops(l)), (c, l)
    g, _ = _pair(d)
    cache = str(tmp_path / "tiles.json")
    res = g.autotune(reps=3, cache=cache)
    assert len(res["cfg"]) == 3 and all(0 <= c < lbm.TILE_CONFIGS for c in res["cfg"])
    g2, _ = _pair(d)
    assert g2.autotune(cache=cache)["cfg"] == res["cfg"]
    g.advance(8)
    for l in range(g.n_levels):
        assert np.array_equal(g.get_pops(l), ref.get_pops(l))


# D3Q19 hierarchy whose level 0 is wide enough for columns that do not meet a periodic
# seam (staged by bulk tensor copies) next to seam columns (staged by plain loads), with
# hole planes under the child box, and a non-periodic level 1 of ragged columns.
D3_WIDE = {"lattice": 19, "coarse_n": (72, 24, 16), "boxes": [((20, 4, 4), (52, 20, 12))], "nu0": 1e-5,
           "init": {"kind": "pulse+vortex", "xc": 30.3, "yc": 11.6, "zc": 7.4, "Rc": 2.5, "A": 1e-3,
                    "swirl": 0.05, "U": (0.06, 0.02, 0.01), "noise": 0.01, "seed": 5}}


def test_d3q19_staged_columns_f64():
    g, o = _pair(D3_WIDE)
    g.advance(5)
    o.advance(5)
    _assert_parity(g, o, 1e-12)


@pytest.mark.parametrize("storage,tol", [("f32", 5e-5), ("f16s", 3e-3)])
def test_d3q19_reduced_precision_against_oracle(storage, tol):
    d = dict(D3_WIDE, storage=storage)
    g, o = _pair(d)
    g.advance(5)
    o.advance(5)
    _assert_parity(g, o, tol)


def test_d3q19_every_chunking_gives_identical_results():
    """The 3-D configurations only change how the z axis is cut into chunks: the
    state is bitwise identical for every one."""
    d = dict(D3_WIDE, storage="f32")
    ref, _ = _pair(d)
    ref.advance(3)
    for c in range(lbm.TILE_CONFIGS):
        g, _ = _pair(d)
        for l in range(g.n_levels):
            g.set_tile_config(l, c)
        g.advance(3)
        for l in range(g.n_levels):
            assert np.array_equal(g.get_pops(l), ref.get_pops(l)), (c, l)


# The interface kernels have two thread mappings (one node per thread for large
# interfaces, one warp segment per node for small ones; AUTO picks by size, so the
# small cases above run segments).  Both must match the oracle.
@pytest.mark.parametrize("mapping", [lbm.IFACE_NODE, lbm.IFACE_SEGMENT])
@pytest.mark.parametrize("case", ["vortex2d", "pulse3lvl", "d3q19"])
def test_interface_mappings_against_oracle_f64(case, mapping):
    if case == "vortex2d":
        d, n = W.vortex2d(), 40
    elif case == "pulse3lvl":
        d, n = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0), 12
    else:
        d, n = D3_WIDE, 4
    g = lbm.Hierarchy(d)
    g.set_interface_mapping(mapping)
    o = O.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
        o.init(l, r, u)
    g.advance(n)
    o.advance(n)
    _assert_parity(g, o, 1e-12)


def test_interface_mappings_agree_f32():
    d = dict(D3_WIDE, storage="f32")
    out = []
    for mapping in (lbm.IFACE_NODE, lbm.IFACE_SEGMENT):
        g, _ = _pair(d)
        g.set_interface_mapping(mapping)
        g.advance(4)
        out.append([g.get_macros(l) for l in range(g.n_levels)])
    for (r0, u0), (r1, u1) in zip(*out):
        assert np.max(np.abs(r0 - r1)) < 1e-6 and np.max(np.abs(u0 - u1)) < 1e-6


def test_f16_storage_shifted_by_mean_flow_equilibrium():
    """FP16 storage of f_i - f_i^eq(1, U) with U the mean flow (u_shift) keeps only the
    perturbation in half precision: it stays within the FP16 bound and is markedly
    closer to the oracle than f_i - w_i, whose mean-flow part takes most of the
    half's precision at Mach 0.1."""
    errs = {}
    for shift in (False, True):
        d = W.vortex2d(storage="f16s")
        if shift:
            d["u_shift"] = tuple(d["init"]["U"])
        g, o = _pair(d)
        g.advance(100)
        o.advance(100)
        errs[shift] = _assert_parity(g, o, 3e-3)
    worst = {k: max(max(er, eu) for er, eu, _ in v) for k, v in errs.items()}
    assert worst[True] < 0.5 * worst[False], worst


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 5e-5), ("f16s", 3e-3)])
def test_d3q19_periodic_extent_not_whole_chunks(storage, tol):
    """Level 0 of 34 x 20 x 16 nodes: its periodic x extent is not a whole number of
    16-byte chunks in FP32 and FP16, so seam columns fill their stage element by
    element; in FP64 (two nodes per chunk) they take 16-byte chunks."""
    d = {"lattice": 19, "coarse_n": (34, 20, 16), "boxes": [((8, 4, 4), (24, 16, 12))], "nu0": 1e-5,
         "storage": storage,
         "init": {"kind": "pulse+vortex", "xc": 15.3, "yc": 9.6, "zc": 7.4, "Rc": 1.5, "A": 1e-3,
                  "swirl": 0.05, "U": (0.05, 0.02, 0.01), "noise": 0.01, "seed": 9}}
    g, o = _pair(d)
    g.advance(4)
    o.advance(4)
    _assert_parity(g, o, tol)
