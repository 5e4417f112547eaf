"""Pins of the oracle's whole hierarchy (Secs. 3.5, 4) against what the paper
and the mathematics fix: uniform flow is a fixed point of every step, the fine
interior does not see the interface before a signal can reach it, a convected
barotropic vortex and a Gaussian acoustic pulse follow their analytic
solutions on a uniform grid, and a two-level run approaches the all-fine run
as both are refined."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_2004_14887_gb300 import workloads as W

CS = 1.0 / math.sqrt(3.0)


def _init_all(h, d):
    for l in range(h.n_levels):
        r, u = W.init_fields(d, l)
        h.init(l, r, u)


@pytest.mark.parametrize("lattice,levels", [(9, 2), (9, 3), (19, 2)])
def test_uniform_flow_is_a_fixed_point(lattice, levels):
    """Equilibrium at uniform (rho, u) is reproduced by streaming, collision,
    Newton at TF nodes, the rebuilds and the interpolations: the flow stays
    uniform to round-off on every level."""
    if lattice == 9:
        boxes = [((8, 8), (24, 24))] + ([((12, 12), (20, 20))] if levels == 3 else [])
        d = {"lattice": 9, "coarse_n": (32, 32), "boxes": boxes, "nu0": 1e-5}
        U = (0.05, -0.03, 0.0)
    else:
        d = {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5}
        U = (0.05, -0.03, 0.02)
    d["init"] = {"kind": "uniform", "rho": 1.0, "U": U}
    h = O.Hierarchy(d)
    _init_all(h, d)
    h.advance(6)
    D = 2 if lattice == 9 else 3
    for l in range(h.n_levels):
        cls = h.node_class(l)
        r, u = h.macros(l)
        m = cls != O.HOLE
        assert np.max(np.abs(r[m] - 1.0)) < 1e-14
        for a in range(D):
            assert np.max(np.abs(u[a][m] - U[a])) < 1e-14


def test_fine_interior_matches_all_fine_run_before_signal_arrives():
    """Domain of dependence: a pulse in the middle of the patch evolves, in the
    part of the fine level that no interface signal can have reached (the
    stencil spans 2 fine nodes per fine step), exactly as on a uniform fine
    grid with the fine relaxation time (Eq. rescTau)."""
    nu0 = 1e-3
    d2 = {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": nu0,
          "init": {"kind": "pulse", "xc": 16.0, "yc": 16.0, "zc": 0.0, "Rc": 1.0, "A": 1e-3, "U": (0.0, 0.0, 0.0)}}
    h2 = O.Hierarchy(d2)
    _init_all(h2, d2)
    # uniform fine grid covering the same domain, level-0 units of half size
    df = {"lattice": 9, "coarse_n": (64, 64), "boxes": [], "nu0": 2 * nu0,
          "init": {"kind": "pulse", "xc": 32.0, "yc": 32.0, "zc": 0.0, "Rc": 2.0, "A": 1e-3, "U": (0.0, 0.0, 0.0)}}
    hf = O.Hierarchy(df)
    r, u = W.init_fields(df, 0)
    hf.init(0, r, u)
    steps = 3
    h2.advance(steps)
    hf.advance(2 * steps)
    r2, u2 = h2.macros(1)
    rf, uf = hf.macros(0)
    n = 33
    r2 = r2.reshape(n, n)
    rf = rf.reshape(64, 64)[16:49, 16:49]
    reach = 2 * (2 * steps) + 1
    core = slice(reach, n - reach)
    assert core.start < core.stop
    assert np.max(np.abs(r2[core, core] - rf[core, core])) < 1e-14
    # and the pulse really moved there: the check is not vacuous
    assert np.max(np.abs(rf[core, core] - 1.0)) > 1e-5


def _vortex_error(n, steps_per_rc=1.0):
    Rc = n / 16.0
    U = 0.1 * CS
    d = {"lattice": 9, "coarse_n": (n, n), "boxes": [], "nu0": 1e-5,
         "init": {"kind": "vortex", "xc": n / 2, "yc": n / 2, "Rc": Rc, "swirl": 0.05, "U": (U, 0.0, 0.0)}}
    h = O.Hierarchy(d)
    _init_all(h, d)
    steps = int(round(steps_per_rc * Rc / U))
    h.advance(steps)
    r, u = h.macros(0)
    x, y, _ = W.level_positions(d, 0)
    _, ux, uy, _ = W.vortex_fields(x.ravel(), y.ravel(), n / 2 + U * steps, n / 2, Rc, 0.05, (U, 0, 0), (n, n))
    eps = 0.05 * CS
    return max(np.max(np.abs(u[0] - ux)), np.max(np.abs(u[1] - uy))) / eps


def test_convected_vortex_second_order():
    """Sec. 4.2: the barotropic vortex of Eq. (init_COVO) is a steady solution
    of the isothermal Euler equations carried by U.  On a uniform periodic grid
    the error after convection by one core radius falls at second order."""
    e = [_vortex_error(n) for n in (32, 64, 128)]
    assert e[2] < 0.05
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0


def _hankel_pulse(r, t, A, Rc, nu):
    def one(rr):
        f = lambda k: k * math.exp(-k * k * Rc * Rc / 2) * math.cos(CS * k * t) * math.exp(-nu * k * k * t) * special.j0(k * rr)  # noqa: E731
        return A * Rc * Rc * integrate.quad(f, 0, 12.0 / Rc, limit=400)[0]
    return np.array([one(rr) for rr in r])


def test_acoustic_pulse_matches_linear_acoustics():
    """Sec. 4.1: a small Gaussian density pulse at rest radiates as 2-D linear
    acoustics, delta rho(r,t) = A Rc^2 int k exp(-k^2 Rc^2/2) cos(c_s k t) J0(k r) dk
    (viscous factor exp(-nu k^2 t)), evaluated by quadrature."""
    n, Rc, A, nu, t = 128, 6.0, 1e-3, 1e-3, 40
    d = {"lattice": 9, "coarse_n": (n, n), "boxes": [], "nu0": nu,
         "init": {"kind": "pulse", "xc": 64.0, "yc": 64.0, "zc": 0.0, "Rc": Rc, "A": A, "U": (0.0, 0.0, 0.0)}}
    h = O.Hierarchy(d)
    _init_all(h, d)
    h.advance(t)
    r, _ = h.macros(0)
    r = r.reshape(n, n)
    line = r[64, 64:120] - 1.0
    ref = _hankel_pulse(np.arange(0, 56, dtype=float), t, A, Rc, nu)
    assert np.max(np.abs(line - ref)) < 0.02 * A
    # the wave front is there (not a vacuous comparison)
    assert np.max(np.abs(ref[20:40])) > 0.1 * A


def _two_level_vs_fine(n, rc_frac=1 / 8, cross=2.0):
    """Vortex crossing a vertical plane interface (the fine level is a slab that
    spans y, as in the paper's Sec. 4.2.1 set-up): 2-level run vs a uniform run
    at the fine spacing, compared on the fine slab."""
    lo, hi = n // 4, 3 * n // 4
    Rc = n * rc_frac
    U = 0.1 * CS
    nu0 = 1e-5 * 32 / n
    ini = {"kind": "vortex", "xc": hi - 0.5 * cross * Rc, "yc": n / 2, "Rc": Rc, "swirl": 0.05, "U": (U, 0.0, 0.0)}
    d2 = {"lattice": 9, "coarse_n": (n, n), "boxes": [((lo, 0), (hi, n))], "nu0": nu0, "init": ini}
    h2 = O.Hierarchy(d2)
    _init_all(h2, d2)
    inif = dict(ini, xc=2 * ini["xc"], yc=2 * ini["yc"], Rc=2 * Rc)
    df = {"lattice": 9, "coarse_n": (2 * n, 2 * n), "boxes": [], "nu0": 2 * nu0, "init": inif}
    hf = O.Hierarchy(df)
    r, u = W.init_fields(df, 0)
    hf.init(0, r, u)
    steps = int(round(cross * Rc / U))
    h2.advance(steps)
    hf.advance(2 * steps)
    _, u2 = h2.macros(1)
    _, uf = hf.macros(0)
    m = 2 * (hi - lo) + 1
    u2 = u2.reshape(2, 2 * n, m)
    uf = uf.reshape(2, 2 * n, 2 * n)[:, :, 2 * lo:2 * hi + 1]
    return np.max(np.abs(u2 - uf)) / (0.05 * CS)


def test_two_level_converges_to_all_fine():
    """Sec. 4.2.1 analogue: the velocity difference between a 2-level DC2 run and
    the all-fine run, on the fine slab after the vortex has crossed the vertical
    interface, falls close to second order when both grids are refined
    (measured ratios 2.8 and 3.5 for 16 -> 32 -> 64 coarse nodes)."""
    e16, e32 = _two_level_vs_fine(16), _two_level_vs_fine(32)
    assert e32 < 0.45 * e16
    assert e32 < 0.01


def test_newton_iterations_at_workload_conditions():
    """Sec. 3.2 reports fewer than three Newton iterations in all cases; with the
    convergence test counted as one more iteration the bound here is 3."""
    d = W.vortex2d(n=64, patch=(16, 48), steps=40)
    h = O.Hierarchy(d)
    _init_all(h, d)
    h.advance(40)
    assert 1 <= h.max_newton_iters <= 3


def test_three_level_pulse_is_stable_and_symmetric():
    """A centred pulse at rest in a symmetric 3-level hierarchy keeps the
    hierarchy's mirror symmetry (x <-> y) and stays bounded."""
    d = {"lattice": 9, "coarse_n": (48, 48), "boxes": [((12, 12), (36, 36)), ((18, 18), (30, 30))], "nu0": 1e-4,
         "init": {"kind": "pulse", "xc": 24.0, "yc": 24.0, "zc": 0.0, "Rc": 1.5, "A": 1e-3, "U": (0.0, 0.0, 0.0)}}
    h = O.Hierarchy(d)
    _init_all(h, d)
    h.advance(30)
    for l in range(3):
        n = h.levels[l]["n"]
        r, u = h.macros(l)
        cls = h.node_class(l).reshape(n[1], n[0])
        r = r.reshape(n[1], n[0])
        m = cls != O.HOLE
        assert np.all(np.abs(r[m] - 1.0) < 2e-3)
        assert np.max(np.abs(np.where(m, r - r.T, 0.0))) < 1e-13


def test_oracle_mirror_symmetry():
    """A pulse at rest at the centre of a mirror-symmetric 3-level D3Q19 hierarchy
    stays symmetric under x -> -x (a symmetry of the lattice, the collision and of
    every interface set and stencil): pins the oracle's sets and stencils against a
    one-sided choice, and is the reference for the full-size GPU symmetry test."""
    d = {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12)), ((6, 6, 6), (10, 10, 10))],
         "nu0": 1e-5, "sigma": 0.98, "dc_variant": 2, "psi_sign": -1, "storage": "f64",
         "init": {"kind": "pulse", "xc": 8.0, "yc": 8.0, "zc": 8.0, "Rc": 1.0, "A": 1e-3, "U": (0.0, 0.0, 0.0)}}
    o = O.Hierarchy(d)
    for l in range(3):
        r, u = W.init_fields(d, l)
        o.init(l, r, u)
    o.advance(4)
    for l in range(3):
        info = o.level_info(l)
        nx, ny, nz = info["n"]
        r, u = o.macros(l)
        R, U = r.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx)
        cls = o.node_class(l).reshape(nz, ny, nx)

        def mirror(a):
            f = a[..., ::-1]
            return np.roll(f, 1, axis=-1) if info["periodic"][0] else f

        assert np.array_equal(cls, mirror(cls))
        active = cls != O.HOLE
        assert np.max(np.abs(R - mirror(R))[active]) < 1e-14
        assert np.max(np.abs(U[0] + mirror(U[0]))[active]) < 1e-14
        assert np.max(np.abs(U[1] - mirror(U[1]))[active]) < 1e-14
    assert np.max(np.abs(R - 1.0)[active]) > 1e-5  # the pulse reached the finest level's nodes


def _slab_pulse_error(n, Rc_f, T, variant):
    """Radial pulse at rest in the middle of a fine slab x in [n/4, 3n/4) that spans
    y (the plane-interface set-up of Sec. 4.1.1, in 2-D): density of the 2-level
    run minus that of the all-fine run on the fine slab after T coarse steps, / A."""
    lo, hi, A = n // 4, n - n // 4, 1e-3
    ini = {"kind": "pulse", "xc": n / 2, "yc": n / 2, "zc": 0.0, "Rc": Rc_f / 2, "A": A, "U": (0.0, 0.0, 0.0)}
    d2 = {"lattice": 9, "coarse_n": (n, n), "boxes": [((lo, 0), (hi, n))], "nu0": 1e-5,
          "dc_variant": variant, "init": ini}
    h2 = O.Hierarchy(d2)
    _init_all(h2, d2)
    h2.advance(T)
    df = {"lattice": 9, "coarse_n": (2 * n, 2 * n), "boxes": [], "nu0": 2e-5,
          "init": dict(ini, xc=float(n), yc=float(n), Rc=Rc_f)}
    hf = O.Hierarchy(df)
    _init_all(hf, df)
    hf.advance(2 * T)
    r2, _ = h2.macros(1)
    rf, _ = hf.macros(0)
    m = 2 * (hi - lo) + 1
    return (r2.reshape(2 * n, m) - rf.reshape(2 * n, 2 * n)[:, 2 * lo:2 * hi + 1]) / A


def test_dc2_reflects_less_than_dc1():
    """Sec. 4.1.1: a pulse crossing plane interfaces is reflected less with DC2 than
    with DC1, which the paper puts down to aliasing of fine content kept by DC1. Here
    the pulse is under-resolved on the coarse grid (R_c = 2.5 fine cells) and the
    reflected wave is measured in the middle half of the slab once it has come back
    from both interfaces: DC2's is 8 % smaller (0.917 of DC1's). The gap closes as the
    pulse is resolved (0.99 at R_c = 5, 1.00 at R_c = 10), as the aliasing reading
    predicts. A swapped (Gamma, gamma) mask reverses the order."""
    n, Rc_f, T = 64, 2.5, 45
    rms = []
    for variant in (1, 2):
        e = _slab_pulse_error(n, Rc_f, T, variant)
        m = e.shape[1]
        c, w = m // 2, m // 4
        rms.append(float(np.sqrt(np.mean(e[:, c - w:c + w + 1] ** 2))))
    assert rms[1] < 0.95 * rms[0]
    # the reflection is there and small: not a vacuous comparison
    assert 1e-4 < rms[1] < 1e-2


def _tf_moment_gap(h, lattice):
    """Largest |moments of the fine TF node - moments of its co-located coarse node| and
    |fine TF moments - X| over every interface of h (populations as stored after a
    coarse step), with the moment scale for reference."""
    c, _ = O.lattice(lattice)
    D = 2 if lattice == 9 else 3
    gap = gx = scale = 0.0
    for l in range(1, h.n_levels):
        fi, ci = h.level_info(l), h.level_info(l - 1)
        ff, fc = h.pops(l), h.pops(l - 1)
        rX, uX = h.macros(l)
        cls = h.node_class(l)
        nf, nc = fi["n"], ci["n"]
        for idx in np.nonzero(cls == O.TFP)[0]:
            x, y, z = idx % nf[0], (idx // nf[0]) % nf[1], idx // (nf[0] * nf[1])
            X = [(p + fi["off"][a]) // 2 - ci["off"][a] for a, p in enumerate((x, y, z))]
            j = X[0] + nc[0] * (X[1] + nc[1] * X[2])
            mf = np.array([ff[:, idx].sum()] + [c[:, a] @ ff[:, idx] for a in range(D)])
            mc = np.array([fc[:, j].sum()] + [c[:, a] @ fc[:, j] for a in range(D)])
            mX = np.array([rX[idx]] + [rX[idx] * uX[a][idx] for a in range(D)])
            gap = max(gap, float(np.max(np.abs(mf - mc))))
            gx = max(gx, float(np.max(np.abs(mf - mX))))
            scale = max(scale, float(np.max(np.abs(mf[1:]))))
    return gap, gx, scale


@pytest.mark.parametrize("lattice,variant", [(9, 2), (9, 1), (19, 2)])
def test_tf_nodes_of_both_levels_carry_X(lattice, variant):
    """Sec. 3.4 (one equilibrium shared by both grids at the interface): after every
    coarse step the fine TF node and the co-located coarse node hold populations with
    one and the same density and momentum, the macros X reported for the TF node (the
    root of Eq. system_fi), to round-off. Pins that both levels collide their TF node
    with X and that the H-RR collision conserves it; a coarse node left with its own
    moments fails (checked by planting that mistake in a copy of the oracle). The
    rebuilds themselves change only non-equilibrium parts and are pinned by the
    two-level convergence and reflection tests."""
    if lattice == 9:
        d = W.vortex2d(n=32, patch=(8, 24), steps=6, levels=3)
    else:
        d = W.vortex3d(n=16, boxes=((4, 12), (6, 10)), steps=3)
    d["dc_variant"] = variant
    h = O.Hierarchy(d)
    _init_all(h, d)
    for _ in range(2):
        h.advance(1)
        gap, gx, scale = _tf_moment_gap(h, lattice)
        assert scale > 1e-3  # the interface carries momentum: not a vacuous check
        assert gap < 1e-14 and gx < 1e-14


def _shear_run(lattice, n, boxes, nu0, T, variant=2, U=1e-3):
    """Shear wave u_x = U sin(2 pi y / n) at rest density on a periodic domain (2-D, or
    3-D uniform in z over n/4 nodes), advanced T coarse steps."""
    D = 2 if lattice == 9 else 3
    d = {"lattice": lattice, "coarse_n": (n, n) if D == 2 else (n, n, n // 4), "boxes": boxes, "nu0": nu0,
         "dc_variant": variant}
    h = O.Hierarchy(d)
    for l in range(h.n_levels):
        info = h.level_info(l)
        nx, ny, nz = info["n"]
        y = np.tile(np.repeat((np.arange(ny) + info["off"][1]) / 2.0 ** l, nx), nz)
        u = np.zeros((D, nx * ny * nz))
        u[0] = U * np.sin(2 * math.pi * y / n)
        h.init(l, np.ones(nx * ny * nz), u)
    h.advance(T)
    return h


def _shear_two_level_vs_fine(lattice, n, nu0, T, variant=2, U=1e-3):
    """max |u_x(2-level) - u_x(all-fine)| / U on the fine slab n/4 <= y < 3n/4 (spanning
    x and z) of a viscous shear wave: the interfaces lie where the wave's curvature is
    largest."""
    lo, hi = n // 4, 3 * n // 4
    box = ((0, lo), (n, hi)) if lattice == 9 else ((0, lo, 0), (n, hi, n // 4))
    h2 = _shear_run(lattice, n, [box], nu0, T, variant, U)
    hf = _shear_run(lattice, 2 * n, [], 2 * nu0, 2 * T, variant, U)
    nx, ny, nz = h2.level_info(1)["n"]
    fx, fy, fz = hf.level_info(0)["n"]
    u2 = h2.macros(1)[1][0].reshape(nz, ny, nx)
    uf = hf.macros(0)[1][0].reshape(fz, fy, fx)[:nz, 2 * lo:2 * hi + 1, :nx]
    return float(np.max(np.abs(u2 - uf))) / U


@pytest.mark.parametrize("variant", [2, 1])
def test_viscous_shear_wave_converges_to_all_fine(variant):
    """Eq. (fneqResc): the non-equilibrium rescaling R = tau_f / (2 tau_c) carries the
    viscous stress across an interface. A shear wave crossing two plane interfaces at
    a viscosity where the non-equilibrium part is large (nu0 = 0.1 at 16 coarse nodes,
    0.05 at 32: the same physical viscosity; decay factor 0.68 over the run) matches
    the all-fine run increasingly well as both grids are refined, at close to second
    order (measured ratios 3.4 for DC2 and 3.1 for DC1; 3.3 and 3.3 once more to 64
    nodes). With R = 1 the DC2 ratio drops to 1.9 and the error at 32 nodes grows 6x
    (checked by planting it in a copy of the oracle). DC2 is 5.6x closer to the
    all-fine run than DC1 here."""
    e16 = _shear_two_level_vs_fine(9, 16, 0.1, 25, variant)
    e32 = _shear_two_level_vs_fine(9, 32, 0.05, 200, variant)
    assert e32 < 0.4 * e16
    assert e32 < (1.5e-3 if variant == 2 else 6e-3)


def test_viscous_shear_wave_d3q19_against_all_fine():
    """The same shear wave on D3Q19 (uniform in z): 1.7e-3 of U against the all-fine
    run at 16 coarse nodes with DC2 (6.2e-3 with R = 1)."""
    assert _shear_two_level_vs_fine(19, 16, 0.1, 25) < 3e-3
