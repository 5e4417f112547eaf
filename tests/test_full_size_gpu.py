"""Full-size checks of the configurations bench.py times, through the C-ABI in the
same launch configuration (CUDA graphs, the bench's storage types), where the oracle
cannot follow the whole run.  They use properties that hold at any size:

* uniform flow is a fixed point of the scheme on every level (equilibrium, zero
  gradients and zero psi in the bulk; the Newton solve returns X; the rescalings of
  Eqs. (rescff) and (rescfc) return f0(X)), so every deviation is rounding;
* a pulse at rest at the centre of a mirror-symmetric hierarchy stays mirror
  symmetric: the oracle is symmetric to 1e-15 on a small replica
  (tests/test_oracle_hierarchy.py::test_oracle_mirror_symmetry), so an index or
  offset error anywhere in a full-size level breaks the symmetry at the scale of the
  pulse amplitude, far above FP32 rounding.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2004_14887_gb300 import lbm  # noqa: E402
from paper_2004_14887_gb300 import workloads as W  # noqa: E402

CS = 1.0 / math.sqrt(3.0)


def _make(d):
    g = lbm.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = W.init_fields(d, l)
        g.init_fields(l, r, u)
    return g


def _macros_dev(g, l):
    N = g.levels[l]["N"]
    rho = torch.empty(N, dtype=torch.float64, device="cuda")
    u = torch.empty((g.D, N), dtype=torch.float64, device="cuda")
    g.get_macros(l, out=(rho, u))
    torch.cuda.synchronize()
    mask = torch.from_numpy(g.node_class(l) != lbm.HOLE).to("cuda")
    return rho, u, mask


def _uniform_deviation(g, U):
    worst = 0.0
    for l in range(g.n_levels):
        rho, u, m = _macros_dev(g, l)
        dev = (rho[m] - 1.0).abs().max().item()
        for a in range(g.D):
            dev = max(dev, (u[a][m] - U[a]).abs().max().item())
        worst = max(worst, dev)
        del rho, u, m
    return worst


def test_vortex3d_full_size_uniform_flow_f32():
    """D3Q19, 3 levels, 256^3 with 128^3 and 64^3 cubes (the vortex3d_3lvl bench
    geometry), FP32 storage: 2 coarse steps = 8 finest-level updates."""
    U = (0.1 * CS, 0.02, -0.01)
    d = dict(W.vortex3d(storage="f32"), init={"kind": "uniform", "rho": 1.0, "U": U})
    g = _make(d)
    g.advance(2)
    g.check_status()
    assert _uniform_deviation(g, U) < 5e-6


def test_slab3d_full_size_uniform_flow_f16s():
    """D3Q19, 3 levels, 512x512x256 with a periodic slab and an inner box (the
    slab3d_3lvl bench geometry, 0.3 G nodes), FP16 shifted storage: 1 coarse step.
    Half precision quantises f - w_i to 2^-11 of itself; the bound matches the small
    uniform-flow test."""
    U = (0.15 * CS, 0.0, 0.0)
    d = dict(W.slab3d(storage="f16s"), init={"kind": "uniform", "rho": 1.0, "U": U})
    g = _make(d)
    g.advance(1)
    g.check_status()
    assert _uniform_deviation(g, U) < 2e-3


def _mirror_x(a, periodic):
    """a[..., x] -> a[..., n - x] (periodic: x -> (n - x) mod n), on the last axis."""
    f = torch.flip(a, dims=(-1,))
    return torch.roll(f, 1, dims=-1) if periodic else f


def test_vortex3d_full_size_mirror_symmetry_f32():
    A = 1e-3
    d = dict(W.vortex3d(storage="f32"),
             init={"kind": "pulse", "xc": 128.0, "yc": 128.0, "zc": 128.0, "Rc": 3.0, "A": A, "U": (0.0, 0.0, 0.0)})
    g = _make(d)
    g.advance(2)
    g.check_status()
    for l in range(g.n_levels):
        nx, ny, nz = (int(v) for v in g.levels[l]["n"])
        per = l == 0  # level 0 is the periodic box; the refined cubes are not periodic
        rho, u, m = _macros_dev(g, l)
        R, Ux, M = rho.view(nz, ny, nx), u[0].view(nz, ny, nx), m.view(nz, ny, nx)
        Rm, Uxm, Mm = _mirror_x(R, per), _mirror_x(Ux, per), _mirror_x(M, per)
        assert torch.equal(M, Mm), l
        assert (R - Rm)[M].abs().max().item() < 2e-2 * A, l
        assert (Ux + Uxm)[M].abs().max().item() < 2e-2 * A, l
        if l == g.n_levels - 1:
            assert (R - 1.0)[M].abs().max().item() > 0.05 * A  # the pulse is there
        del rho, u, m


def test_batch2d_full_size_uniform_flow_f32():
    """The 96 hierarchies of the batch2d bench workload, each with its own uniform
    flow, advanced together in the persistent launch: every member stays uniform."""
    descs = W.batch2d(storage="f32")
    rng = np.random.default_rng(7)
    Us = []
    for d in descs:
        U = (float(rng.uniform(-0.08, 0.08)), float(rng.uniform(-0.08, 0.08)), 0.0)
        d["init"] = {"kind": "uniform", "rho": 1.0, "U": U}
        Us.append(U)
    b = lbm.Batch(descs)
    for d, mbr in zip(descs, b.members):
        for l in range(mbr.n_levels):
            r, u = W.init_fields(d, l)
            mbr.init_fields(l, r, u)
    b.advance(2)
    b.check_status()
    worst = max(_uniform_deviation(mbr, U) for mbr, U in zip(b.members, Us))
    assert worst < 5e-6
