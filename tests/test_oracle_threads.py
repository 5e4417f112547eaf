"""The OpenMP build of the oracle against its plain build.

Every per-node loop of a step writes only its own node (and, in the coarse
rebuild of Eq. (rescfc), the one coarse node co-located with it), so sharing the
nodes out over threads must not change a single bit: populations, Newton counts
and update counts are compared exactly after several coarse steps of a 3-level
D2Q9 hierarchy and of a 3-level D3Q19 slab hierarchy.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_14887_gb300 import workloads as W


def _run(d, steps, threaded):
    o = O.Hierarchy(d, threaded=threaded)
    for l in range(o.n_levels):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    o.advance(steps)
    return [o.pops(l) for l in range(o.n_levels)], o.max_newton_iters, o.node_updates


@pytest.mark.parametrize("case", ["d2q9_3lvl", "d3q19_slab"])
def test_threaded_oracle_is_bitwise_equal(case):
    if case == "d2q9_3lvl":
        d, n = W.pulse2d(n=64, boxes=((16, 48), (24, 40)), Rc_finest=3.0), 6
    else:
        d, n = {"lattice": 19, "coarse_n": (16, 16, 24), "boxes": [((0, 0, 6), (16, 16, 18)), ((4, 4, 9), (12, 12, 15))],
                "nu0": 1e-5, "init": {"kind": "pulse+vortex", "xc": 8.2, "yc": 7.9, "zc": 12.1, "Rc": 1.5, "A": 1e-3,
                                      "swirl": 0.05, "U": (0.05, 0.0, 0.0)}}, 2
    O.threads(4)
    fa, na, ua = _run(d, n, False)
    fb, nb, ub = _run(d, n, True)
    assert na == nb and ua == ub
    for a, b in zip(fa, fb):
        assert np.array_equal(a, b)
