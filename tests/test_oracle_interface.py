"""Pins of the oracle's direct-coupling interface pieces (Sec. 3 and App. B):
population sets, Newton solve, temporal and spatial interpolation weights."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _bits(mask, q):
    return {i for i in range(q) if (mask >> i) & 1}


def _grid(s):
    """'110/110/110' rows dy=+1,0,-1, columns dx=-1,0,+1 -> array [dy+1][dx+1]."""
    rows = s.split("/")
    g = np.zeros((3, 3), np.uint8)
    for r, dy in zip(rows, (1, 0, -1)):
        for ch, dx in zip(r, (-1, 0, 1)):
            g[dy + 1, dx + 1] = ch == "1"
    return g


def _golden_sets():
    out = []
    for line in open(os.path.join(GOLDEN, "sets_fig1_appB.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, occf, occc, P, Qf, Mf, _src = [t.strip() for t in line.split("|")]
        sets = [{int(v) for v in t.split(",")} for t in (P, Qf, Mf)]
        out.append((name, _grid(occf), _grid(occc), *sets))
    return out


@pytest.mark.parametrize("case", _golden_sets(), ids=lambda c: c[0])
def test_population_sets_match_paper(case):
    """Sec. 3.2 (Fig. 1) and App. B (Figs. corner1, corner2): the set rule applied
    to the drawn grids gives exactly the printed P, Q^f and M^f."""
    name, occf, occc, P, Qf, Mf = case
    kf, kc = O.known_from_occupancy(9, occf, occc)
    fk, ck = _bits(kf, 9), _bits(kc, 9)
    assert fk & ck == P
    assert fk - ck == Qf
    assert set(range(9)) - fk == Mf


def test_hierarchy_sets_on_patch_faces_and_corners():
    """A 2-level box patch: the right face TF nodes see the Fig. 1 sets, the
    top-right corner the concave-corner sets of App. B; hanging nodes miss the
    same populations as the TF nodes of their face."""
    d = {"lattice": 9, "coarse_n": (32, 32), "boxes": [((8, 8), (24, 24))], "nu0": 1e-5}
    h = O.Hierarchy(d)
    lv = h.levels[1]
    n = lv["n"][0]
    cls = h.node_class(1).reshape(lv["n"][1], n)
    kf, kc = (m.reshape(lv["n"][1], n) for m in h.known_masks(1))
    # right face, mid-height TF (fine interior to the left, as Fig. 1)
    y = 10
    assert cls[y, n - 1] == O.TFP
    fk, ck = _bits(kf[y, n - 1], 9), _bits(kc[y, n - 1], 9)
    assert set(range(9)) - fk == {4, 5, 6} and fk & ck == {0, 3, 7} and fk - ck == {1, 2, 8}
    assert cls[y + 1, n - 1] == O.IE and set(range(9)) - _bits(kf[y + 1, n - 1], 9) == {4, 5, 6}
    # top-right corner: fine region is the lower-left quadrant, as App. B Fig. corner1
    fk, ck = _bits(kf[n - 1, n - 1], 9), _bits(kc[n - 1, n - 1], 9)
    assert fk & ck == {0, 1, 3} and fk - ck == {2} and set(range(9)) - fk == {4, 5, 6, 7, 8}
    # class counts: a 33x33 fine box has 64 boundary nodes, half of them TF
    assert (cls == O.TFP).sum() == 64 and (cls == O.IE).sum() == 64
    # the coarse level holds the matching TF nodes on the patch outline, the hole inside
    c0 = h.node_class(0).reshape(32, 32)
    assert (c0 == O.TFC).sum() == 64 and (c0 == O.HOLE).sum() == 15 * 15


def test_d3q19_face_edge_corner_sets():
    """3-D extension (App. B states it is direct): on a face the fine level misses the
    5 populations coming from outside, on an edge 9, on a corner 12 (D3Q19); every
    missing population is known on the coarse level."""
    d = {"lattice": 19, "coarse_n": (16, 16, 16), "boxes": [((4, 4, 4), (12, 12, 12))], "nu0": 1e-5}
    h = O.Hierarchy(d)
    n = h.levels[1]["n"][0]
    cls = h.node_class(1).reshape(n, n, n)
    kf, kc = (m.reshape(n, n, n) for m in h.known_masks(1))
    full = (1 << 19) - 1
    for (z, y, x), nmiss in [((4, 6, 0), 5), ((4, 0, 0), 9), ((0, 0, 0), 12)]:
        assert cls[z, y, x] == O.TFP
        assert 19 - bin(int(kf[z, y, x])).count("1") == nmiss
        assert int(kf[z, y, x]) | int(kc[z, y, x]) == full


def test_tempint_weights_golden_and_exact_on_quadratics():
    """Eq. (TempInt): weights -1/8, 3/4, 3/8 (printed), exact for any quadratic
    through t - dt^c, t, t + dt^c evaluated at t + dt^f (reading R5)."""
    gold = {}
    for line in open(os.path.join(GOLDEN, "interp_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        gold[k] = np.array([float(x) for x in v])
    w = O.tempint_weights()
    assert np.array_equal(w, gold["tempint"])
    rng = np.random.default_rng(0)
    for _ in range(5):
        a, b, c = rng.normal(size=3)
        g = lambda t: a + b * t + c * t * t  # noqa: E731
        assert abs(w @ np.array([g(-2.0), g(0.0), g(2.0)]) - g(1.0)) < 1e-14
    wc, wo = O.lagrange4_weights(False), O.lagrange4_weights(True)
    assert np.array_equal(wc, gold["lagrange4_centred"]) and np.array_equal(wo, gold["lagrange4_onesided"])
    for _ in range(5):
        p = rng.normal(size=4)
        g = lambda x: p[0] + p[1] * x + p[2] * x * x + p[3] * x ** 3  # noqa: E731
        assert abs(wc @ np.array([g(-1), g(0), g(1), g(2)]) - g(0.5)) < 1e-13
        assert abs(wo @ np.array([g(0), g(1), g(2), g(3)]) - g(0.5)) < 1e-13


def _dc2_gamma(q, R, coarse):
    return np.where(coarse, R, 1.0)


@pytest.mark.parametrize("q", [9, 19])
def test_newton_jacobian_matches_finite_differences(q):
    """Eq. (system_fi): the analytic Jacobian equals central differences of F."""
    rng = np.random.default_rng(1)
    D = 2 if q == 9 else 3
    c, w = O.lattice(q)
    fhat = O.feq(q, 1.02, [0.05, -0.03, 0.02][:D] + [0] * (3 - D)) * (1 + 0.01 * rng.normal(size=q))
    gam = _dc2_gamma(q, 0.9, rng.random(q) < 0.5)
    X = np.array([1.01, 0.04, -0.02, 0.01][: D + 1])
    F, J = O.newton_system(q, fhat, gam, X)
    h = 1e-6
    for k in range(D + 1):
        dx = np.zeros(D + 1)
        dx[k] = h
        Fp, _ = O.newton_system(q, fhat, gam, X + dx)
        Fm, _ = O.newton_system(q, fhat, gam, X - dx)
        assert np.allclose((Fp - Fm) / (2 * h), J[:, k], atol=1e-9)


@pytest.mark.parametrize("q", [9, 19])
def test_newton_unit_gamma_gives_plain_moments(q):
    """With Gamma = 1 on every population the system is the definition of the
    moments: the first iterate from the plain moments already satisfies it."""
    rng = np.random.default_rng(2)
    c, _ = O.lattice(q)
    D = 2 if q == 9 else 3
    fhat = O.feq(q, 1.0, [0.05, 0.02, -0.01][:D] + [0] * (3 - D)) * (1 + 0.01 * rng.normal(size=q))
    X, it = O.newton(q, fhat, np.ones(q))
    assert it == 1
    assert abs(X[0] - fhat.sum()) < 1e-15
    assert np.allclose(X[1:], fhat @ c[:, :D] / fhat.sum(), atol=1e-16)


@pytest.mark.parametrize("q", [9, 19])
def test_newton_recovers_manufactured_root(q):
    """A root X* is planted: fhat = f0(X*) + g with sum Gamma Phi g = 0.  Newton
    recovers X* to 1e-14 in at most 3 iterations (Sec. 3.2 reports fewer than
    three), with quadratic convergence of the residual."""
    rng = np.random.default_rng(3)
    c, _ = O.lattice(q)
    D = 2 if q == 9 else 3
    Phi = np.concatenate([np.ones((q, 1)), c[:, :D]], axis=1)
    for trial in range(10):
        Xs = np.concatenate([[rng.uniform(0.98, 1.02)], rng.uniform(-0.08, 0.08, D)])
        gam = _dc2_gamma(q, rng.uniform(0.5, 1.0), rng.random(q) < 0.5)
        g = 1e-3 * rng.normal(size=q)
        A = (gam[:, None] * Phi).T  # (D+1, q)
        g = g - A.T @ np.linalg.solve(A @ A.T, A @ g)  # project onto the null space
        fhat = O.feq(q, Xs[0], list(Xs[1:]) + [0] * (3 - D)) + g
        X, it = O.newton(q, fhat, gam)
        assert 1 <= it <= 3
        assert np.max(np.abs(X - Xs)) < 1e-14
    # quadratic convergence: error after one step of a displaced start ~ error^2
    F0, J0 = O.newton_system(q, fhat, gam, Xs + 1e-3)
    X1 = Xs + 1e-3 - np.linalg.solve(J0, F0)
    assert np.max(np.abs(X1 - Xs)) < 50 * 1e-6


def test_interface_gradients_match_taylor_green_derivatives():
    """Sec. 3.3, Eqs. (PijResc) and (PSIResc), readings R8 and R10: the strain rate S
    and C_ab = sum_g d_g Psi_abg supplied to the interface nodes after one coarse step
    of a Taylor-Green vortex (u_x = U sin kx cos ky, u_y = -U cos kx sin ky, a steady
    inviscid flow) equal the analytic derivatives in each level's lattice units: x 1/2
    at fine TF and hanging nodes, x 1 at the co-located coarse nodes. Measured worst
    errors: 1.4 % of U k on S_xx and S_yy, 2.8 % on S_xy, 1.0 % of 3 U^3 k on C (the
    coarse and fine sides' start-up transients differ; the errors halve with each
    doubling of n). The fine-level S with its factor 1/2 lost (planted in a copy of the
    oracle) is 72 % off; a wrong sign or swapped axes is as far off."""
    n, U = 64, 1e-3
    k = 2 * math.pi / n
    lo, hi = n // 4, 3 * n // 4
    h = O.Hierarchy({"lattice": 9, "coarse_n": (n, n), "boxes": [((lo, lo), (hi, hi))], "nu0": 1e-5})

    def coords(l):
        # the vortex cells are shifted by n/8 so that the outline does not sit on the
        # zeros of S and C
        info = h.level_info(l)
        nx, ny, _ = info["n"]
        s = 2.0 ** l
        return (np.tile((np.arange(nx) + info["off"][0]) / s + n / 8, ny),
                np.repeat((np.arange(ny) + info["off"][1]) / s + n / 8, nx))

    for l in range(2):
        X, Y = coords(l)
        u = np.stack([U * np.sin(k * X) * np.cos(k * Y), -U * np.cos(k * X) * np.sin(k * Y)])
        h.init(l, np.ones(X.size), u)
    h.advance(1)
    checked = 0
    for l, scale, classes in [(1, 0.5, (O.TFP, O.IE)), (0, 1.0, (O.TFC,))]:
        X, Y = coords(l)
        S, Cg = h.gradients(l)
        m = np.isin(h.node_class(l), classes)
        cx, sx, cy, sy = np.cos(k * X), np.sin(k * X), np.cos(k * Y), np.sin(k * Y)
        sxx = U * k * cx * cy
        want = {0: (S[0], sxx), 1: (S[1], -sxx), 3: (S[3], 0.0 * X)}
        for _, (got, w) in want.items():
            assert np.max(np.abs(got[m] - scale * w[m])) < 0.04 * scale * U * k
        c3 = 3 * U ** 3 * k
        cxx, cyy = c3 * sx ** 2 * cx * cy ** 3, -c3 * cx ** 3 * sy ** 2 * cy
        assert np.max(np.abs(Cg[0][m] - scale * cxx[m])) < 0.04 * scale * c3
        assert np.max(np.abs(Cg[1][m] - scale * cyy[m])) < 0.04 * scale * c3
        checked += int(m.sum())
    assert checked == 12 * (hi - lo)  # fine outline: 8 (hi - lo) TF and hanging nodes; coarse: 4 (hi - lo)


def test_interface_gradients_match_taylor_green_derivatives_d3q19():
    """The 3-D counterpart on D3Q19 (faces, edges, corners and the face-centre hanging
    nodes of reading R10): S and C at TF, hanging and co-located coarse nodes after one
    coarse step of u = U (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0) against its
    analytic derivatives, C_ab = sum_g d_g Psi_abg with the Psi components of reading
    R3 differentiated symbolically. Measured worst errors at 32 coarse nodes: 4.9 % of
    U k on S, 3.9 % of 3 U^3 k on C, both at TF nodes next to the box edges, where the
    start-up transient leaves a small w; the median S error is 0.3 %."""
    sp = pytest.importorskip("sympy")
    n, U = 32, 1e-3
    lo, hi = n // 4, 3 * n // 4
    X = sp.symbols("x y z")
    kk, sh = 2 * sp.pi / n, sp.Rational(n, 8)
    s = [sp.sin(kk * (v + sh)) for v in X]
    c = [sp.cos(kk * (v + sh)) for v in X]
    u = [U * s[0] * c[1] * c[2], -U * c[0] * s[1] * c[2], sp.Integer(0)]

    def psi(a, b, g):
        idx = sorted((a, b, g))
        if idx[0] == idx[2]:
            return u[idx[0]] ** 3
        if len(set(idx)) == 3:
            return u[0] * u[1] * u[2]
        rep = idx[1]
        single = idx[0] if idx[2] == rep else idx[2]
        third = 3 - rep - single
        return sp.Rational(1, 2) * u[single] * u[third] ** 2

    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    S_an = [sp.lambdify(X, (sp.diff(u[a], X[b]) + sp.diff(u[b], X[a])) / 2, "numpy") for a, b in pairs]
    C_an = [sp.lambdify(X, sum(sp.diff(psi(a, b, g), X[g]) for g in range(3)), "numpy") for a, b in pairs]
    u_an = [sp.lambdify(X, e, "numpy") for e in u]
    h = O.Hierarchy({"lattice": 19, "coarse_n": (n, n, n), "boxes": [((lo,) * 3, (hi,) * 3)], "nu0": 1e-5})

    def coords(l):
        info = h.level_info(l)
        g = [(np.arange(info["n"][a]) + info["off"][a]) / 2.0 ** l for a in range(3)]
        Z, Y, Xc = np.meshgrid(g[2], g[1], g[0], indexing="ij")
        return Xc.ravel(), Y.ravel(), Z.ravel()

    def ev(f, p):
        return np.broadcast_to(f(*p), p[0].shape)

    for l in range(2):
        p = coords(l)
        h.init(l, np.ones(p[0].size), np.stack([ev(f, p) for f in u_an]))
    h.advance(1)
    k = 2 * math.pi / n
    for l, scale, classes in [(1, 0.5, (O.TFP, O.IE)), (0, 1.0, (O.TFC,))]:
        p = coords(l)
        S, Cg = h.gradients(l)
        m = np.isin(h.node_class(l), classes)
        assert m.any()
        for i in range(6):
            assert np.max(np.abs(S[i][m] - scale * ev(S_an[i], p)[m])) < 0.08 * scale * U * k
            assert np.max(np.abs(Cg[i][m] - scale * ev(C_an[i], p)[m])) < 0.06 * scale * 3 * U ** 3 * k
