"""Pins of the oracle on staircase refinement interfaces (paper Sec. 4.1.2 circular
interface, Sec. 4.2.2 inclined interface, App. B corners): a refined region given as a
mask of parent cells instead of a box.

* a mask that refines the whole box is the box hierarchy, bit for bit;
* the re-entrant corner of an L-shaped region carries the convex-corner sets of App. B
  (Fig. corner2), its outer corners the concave-corner sets (Fig. corner1);
* every hanging-node stencil is a collinear set of TF nodes along the node's odd axis,
  exact on cubics (4 points) or on linear fields (2 points, reading R15), and the
  stencils of a symmetric region are the mirror images of each other;
* a uniform flow is a fixed point of staircase hierarchies;
* a pulse centred in a disk-shaped region keeps the square's symmetries;
* a staircase 2-level run approaches the all-fine run as both are refined.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_14887_gb300 import workloads as W


def _bits(m, q=9):
    return {i for i in range(q) if (int(m) >> i) & 1}


def _run(d, steps, threaded=True):
    o = O.Hierarchy(d, threaded=threaded)
    for l in range(o.n_levels):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    o.advance(steps)
    return o


def test_full_mask_is_the_box_bit_for_bit():
    d = W.vortex2d(n=32, patch=(8, 24), steps=6)
    dm = dict(d, masks=[None, np.ones((16, 16), np.uint8)])
    a, b = _run(d, 6), _run(dm, 6)
    for l in range(2):
        assert np.array_equal(a.node_class(l), b.node_class(l))
        assert np.array_equal(a.pops(l), b.pops(l))


def _l_shape():
    """Box [8, 24)^2 of a 32^2 coarse grid with its top-right quadrant left coarse."""
    m = np.ones((16, 16), np.uint8)
    m[8:, 8:] = 0  # cells x >= 16, y >= 16
    return {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "masks": [None, m], "nu0": 1e-5}


def test_app_b_corner_sets_on_an_l_shaped_region():
    h = O.Hierarchy(_l_shape())
    lv = h.levels[1]
    nx, ny = lv["n"][0], lv["n"][1]
    cls = h.node_class(1).reshape(ny, nx)
    kf, kc = (m.reshape(ny, nx) for m in h.known_masks(1))
    off = lv["off"]
    # re-entrant corner at fine (32, 32): fine region in three quadrants, Fig. corner2
    j, i = 32 - off[1], 32 - off[0]
    assert cls[j, i] == O.TFP
    fk, ck = _bits(kf[j, i]), _bits(kc[j, i])
    assert fk & ck == {0, 5, 7} and fk - ck == {1, 2, 3, 4, 8} and set(range(9)) - fk == {6}
    # outer corner at fine (32, 48): the fine region is the lower-left quadrant, Fig. corner1
    j, i = 32 - off[1], 48 - off[0]
    assert cls[j, i] == O.TFP
    fk, ck = _bits(kf[j, i]), _bits(kc[j, i])
    assert fk & ck == {0, 1, 3} and fk - ck == {2} and set(range(9)) - fk == {4, 5, 6, 7, 8}
    # nodes of the cut quadrant are not nodes of the fine level; coarse nodes inside it
    # are bulk, those on its edges co-located with fine TF nodes
    assert cls[40 - off[1], 40 - off[0]] == O.HOLE
    c0 = h.node_class(0).reshape(32, 32)
    assert c0[20, 20] == O.BULK and c0[16, 20] == O.TFC and c0[12, 12] == O.HOLE


@pytest.mark.parametrize("make", [W.pulse_circle, W.vortex_inclined, _l_shape], ids=["circle", "inclined", "L"])
def test_hanging_node_stencils_are_collinear_tf_sets_exact_on_polynomials(make):
    d = make() if make is not _l_shape else _l_shape()
    h = O.Hierarchy(d)
    lv = h.levels[1]
    cls = h.node_class(1)
    off = lv["off"]
    nx = lv["n"][0]
    n4 = n2 = 0
    for idx in np.nonzero(cls == O.IE)[0]:
        p = np.array([idx % nx + off[0], idx // nx + off[1], 0])
        pts, w = h.ie_stencil(1, idx)
        odd = [a for a in range(2) if p[a] % 2]
        assert len(odd) == 1
        a = odd[0]
        b = 1 - a
        assert np.all(pts[:, b] == p[b]) and np.all(pts[:, 2] == 0)  # on the node's line
        for q in pts:  # every stencil node is a TF node of the level
            j = (q[0] - off[0]) + nx * (q[1] - off[1])
            assert cls[j] == O.TFP
        t = (pts[:, a] - p[a]).astype(float)
        assert abs(w.sum() - 1.0) < 1e-15
        deg = 3 if len(w) == 4 else 1
        for k in range(1, deg + 1):  # exact on polynomials of the stencil's degree
            assert abs(np.dot(w, t ** k)) < 1e-13
        if len(w) == 4:
            n4 += 1
        else:
            assert len(w) == 2 and sorted(t) == [-1.0, 1.0]
            n2 += 1
    assert n4 > 0
    if make is W.pulse_circle:
        assert n2 > 0  # the circle has steps of one coarse cell
    if make is _l_shape:
        # straight edges of at least 8 coarse cells: every hanging node has a complete
        # centred or one-sided 4-point set (reading R10 next to the corners)
        assert n2 == 0


def test_box_corner_hanging_nodes_take_the_one_sided_stencil():
    """Reading R10 on a box: the hanging node next to a corner interpolates from
    (-1, 1, 3, 5) with weights (5, 15, -5, 1)/16, the others from (-3, -1, 1, 3) with
    (-1, 9, 9, -1)/16."""
    d = {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": 1e-5}
    h = O.Hierarchy(d)
    lv = h.levels[1]
    off, nx = lv["off"], lv["n"][0]
    # bottom face y = 16 (fine), hanging nodes at x = 17 (next to the corner) and 21
    for x, offs, w in ((17, (-1, 1, 3, 5), (5, 15, -5, 1)), (21, (-3, -1, 1, 3), (-1, 9, 9, -1))):
        idx = (x - off[0]) + nx * (16 - off[1])
        pts, ws = h.ie_stencil(1, idx)
        got = sorted(zip((pts[:, 0] - x).tolist(), (16 * ws).tolist()))
        assert got == sorted(zip(offs, map(float, w)))


def test_circle_stencils_are_mirror_images():
    d = W.pulse_circle()
    h = O.Hierarchy(d)
    lv = h.levels[1]
    nx, ny = lv["n"][0], lv["n"][1]
    assert nx == ny
    cls = h.node_class(1).reshape(ny, nx)
    assert np.array_equal(cls, cls[:, ::-1]) and np.array_equal(cls, cls[::-1, :]) and np.array_equal(cls, cls.T)
    off = lv["off"][0]
    mirror = 2 * off + nx - 1  # x -> mirror - x on fine global coordinates
    for j, i in zip(*np.nonzero(cls == O.IE)):
        pts, w = h.ie_stencil(1, j * nx + i)
        pm, wm = h.ie_stencil(1, j * nx + (nx - 1 - i))
        ref = sorted(zip((mirror - pts[:, 0]).tolist(), pts[:, 1].tolist(), w.tolist()))
        got = sorted(zip(pm[:, 0].tolist(), pm[:, 1].tolist(), wm.tolist()))
        assert ref == got


@pytest.mark.parametrize("make", [W.pulse_circle, W.vortex_inclined], ids=["circle", "inclined"])
def test_uniform_flow_is_a_fixed_point_of_staircase_hierarchies(make):
    d = make()
    d["init"] = {"kind": "uniform", "rho": 1.0, "U": (0.04, -0.03, 0.0)}
    o = _run(d, 10)
    for l in range(2):
        m = o.node_class(l) != O.HOLE
        r, u = o.macros(l)
        assert np.max(np.abs(r[m] - 1.0)) < 1e-14
        assert np.max(np.abs(u[0, m] - 0.04)) < 1e-14 and np.max(np.abs(u[1, m] + 0.03)) < 1e-14


def test_pulse_in_a_disk_region_keeps_the_square_symmetries():
    """A pulse at rest at the centre of the circular region: the disk of refined cells
    and the centred stencils are symmetric under the square's reflections, so the
    density stays symmetric to round-off on both levels."""
    d = W.pulse_circle(steps=24)
    d["init"] = dict(d["init"], xc=32.0, yc=32.0, U=(0.0, 0.0, 0.0))
    o = _run(d, 24)
    amp = 0.0
    for l in range(2):
        lv = o.levels[l]
        ny, nx = lv["n"][1], lv["n"][0]
        r = o.macros(l)[0].reshape(ny, nx)
        if l == 0:
            # periodic 64^2 grid centred on node 32: x -> 64 - x
            r = np.roll(r, -32, axis=(0, 1))
            r = np.roll(r[::-1, ::-1], 1, axis=(0, 1))  # reflect about node 0 then realign
            base = np.roll(o.macros(0)[0].reshape(ny, nx), -32, axis=(0, 1))
            imgs = [r, base.T]
            ref = base
        else:
            ref = r
            imgs = [r[::-1, :], r[:, ::-1], r.T]
        m = ref != 0.0
        amp = max(amp, np.max(np.abs(ref[m] - 1.0)))
        for im in imgs:
            # round-off on densities near 1; a stencil that breaks the symmetry would
            # leave differences of the order of the signal (1e-5 here)
            assert np.max(np.abs(im[m] - ref[m])) < 1e-12
    assert amp > 1e-5


def _all_fine(d):
    f = 2
    u = dict(d)
    u["boxes"] = []
    u.pop("masks", None)
    u["coarse_n"] = tuple(c * f for c in d["coarse_n"])
    u["nu0"] = d["nu0"] * f
    u["init"] = dict(d["init"], xc=d["init"]["xc"] * f, yc=d["init"]["yc"] * f, Rc=d["init"]["Rc"] * f)
    return u


def test_circular_interface_run_approaches_the_all_fine_run():
    """The pulse of Sec. 4.1.2 crossing the circular staircase: the fine level of the
    2-level run against an all-fine run over the same physical time, at two
    resolutions (every length doubled): the error shrinks."""
    errs = []
    for s in (1, 2):
        n = 32 * s
        lo, hi = 6 * s, 26 * s
        steps = 16 * s
        d = W.pulse_circle(n=n, box=((lo, lo), (hi, hi)), radius=8.0 * s, Rc_fine=2.0 * s, A=1e-3, steps=steps)
        d["init"] = dict(d["init"], xc=n / 2, yc=n / 2)
        o = _run(d, steps)
        ou = _run(_all_fine(d), 2 * steps)
        lv = o.levels[1]
        nx, ny = lv["n"][0], lv["n"][1]
        rf = o.macros(1)[0].reshape(ny, nx)
        ru = ou.macros(0)[0].reshape(2 * n, 2 * n)
        off = lv["off"]
        sub = ru[off[1]:off[1] + ny, off[0]:off[0] + nx]
        m = o.node_class(1).reshape(ny, nx) != O.HOLE
        errs.append(np.max(np.abs(rf[m] - sub[m])) / 1e-3)
    print("circular interface, fine-level error vs all-fine (relative to A):", errs)
    assert errs[1] < errs[0] / 1.5
