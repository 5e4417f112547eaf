"""Pins of the oracle's D3Q19 hanging-node stencils on a refined box (reading R10:
4-point 1-D Lagrange along each odd axis, one-sided next to the box's edges, tensor
order for face nodes odd along both in-face axes; Sec. 3.2, steps 2g / 3e).

* every stencil point is a TF node of the level in the node's face (or edge) plane;
* the weights reproduce every monomial of degree <= 3 per odd axis exactly (a plain
  Lagrange property: a dropped or shifted point, a wrong weight or a transposed axis
  fails it);
* along each odd axis the offsets are the centred (-3, -1, 1, 3) set or, next to an
  edge of the box, the one-sided set on the same line;
* the stencils of a box centred in the domain are mirror images of each other.
"""
import itertools

import numpy as np

from oracle import oracle as O


def _box_hierarchy():
    return {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5}


def _ie_nodes(h, l):
    lv = h.levels[l]
    nx, ny, _ = lv["n"]
    off = np.array(lv["off"])
    cls = h.node_class(l)
    for idx in np.nonzero(cls == O.IE)[0]:
        p = np.array([idx % nx, (idx // nx) % ny, idx // (nx * ny)]) + off
        yield int(idx), p


def test_d3q19_hanging_node_stencils_are_tensor_lagrange_sets():
    h = O.Hierarchy(_box_hierarchy())
    lv = h.levels[1]
    nx, ny, nz = lv["n"]
    off = np.array(lv["off"])
    cls = h.node_class(1)
    counts = {1: 0, 2: 0}
    one_sided = 0
    for idx, p in _ie_nodes(h, 1):
        pts, w = h.ie_stencil(1, idx)
        odd = [a for a in range(3) if p[a] % 2]
        assert len(odd) in (1, 2), (p, odd)
        counts[len(odd)] += 1
        assert len(w) == 4 ** len(odd)
        for b in range(3):
            if b not in odd:
                assert np.all(pts[:, b] == p[b])  # in the node's plane or line
        for q in pts:  # TF nodes of the level
            j = (q[0] - off[0]) + nx * ((q[1] - off[1]) + ny * (q[2] - off[2]))
            assert cls[j] == O.TFP
        t = (pts - p).astype(float)
        for ks in itertools.product(range(4), repeat=len(odd)):
            mono = np.prod([t[:, a] ** k for a, k in zip(odd, ks)], axis=0)
            want = 1.0 if all(k == 0 for k in ks) else 0.0
            assert abs(np.dot(w, mono) - want) < 1e-12, (p, ks)
        for a in odd:
            offs = sorted(set((pts[:, a] - p[a]).tolist()))
            assert offs in ([-3, -1, 1, 3], [-1, 1, 3, 5], [-5, -3, -1, 1]), (p, a, offs)
            one_sided += offs != [-3, -1, 1, 3]
    assert counts[1] > 0 and counts[2] > 0 and one_sided > 0
    assert nx == ny == nz


def test_d3q19_stencils_of_a_centred_box_are_mirror_images():
    h = O.Hierarchy(_box_hierarchy())
    lv = h.levels[1]
    nx, ny, _ = lv["n"]
    off = np.array(lv["off"])
    mirror = 2 * off[0] + nx - 1  # x -> mirror - x in fine global coordinates
    nodes = {tuple(p): idx for idx, p in _ie_nodes(h, 1)}
    for p, idx in nodes.items():
        q = (mirror - p[0], p[1], p[2])
        assert q in nodes
        pts, w = h.ie_stencil(1, idx)
        pm, wm = h.ie_stencil(1, nodes[q])
        ref = sorted(zip((mirror - pts[:, 0]).tolist(), pts[:, 1].tolist(), pts[:, 2].tolist(), w.tolist()))
        got = sorted(zip(pm[:, 0].tolist(), pm[:, 1].tolist(), pm[:, 2].tolist(), wm.tolist()))
        assert ref == got
