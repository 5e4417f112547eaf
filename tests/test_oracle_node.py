"""Pins of the oracle's node-local arithmetic (Sec. 2 and App. A of the paper)
against closed forms, invariants and properties the paper fixes.

Each test would fail for a plausible slip in the oracle: a dropped Hermite
term, a wrong factor of 2 on off-diagonals, a sign error in psi, a transposed
index in the recursive third-order coefficients.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O

CS2 = 1.0 / 3.0
LATTICES = [9, 19]


def _D(q):
    return 2 if q == 9 else 3


def _rand_state(rng, q, mach=0.15):
    D = _D(q)
    rho = rng.uniform(0.9, 1.1)
    u = np.zeros(3)
    u[:D] = rng.uniform(-mach, mach, D) * math.sqrt(CS2)
    return rho, u


@pytest.mark.parametrize("q", LATTICES)
def test_lattice_isotropy(q):
    """Sec. 2: weights and velocities form a lattice with c_s^2 = 1/3 and
    isotropic moments up to 4th order (Eqs. xi_i, w_i)."""
    c, w = O.lattice(q)
    D = _D(q)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2[:D, :D], CS2 * np.eye(D), atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    for a, b, cc, d in itertools.product(range(D), repeat=4):
        iso = CS2 * CS2 * ((a == b) * (cc == d) + (a == cc) * (b == d) + (a == d) * (b == cc))
        assert abs(M4[a, b, cc, d] - iso) < 1e-15
    # every velocity has its opposite
    for i in range(q):
        assert any((c[j] == -c[i]).all() for j in range(q))


def test_d2q9_numbering_matches_fig1():
    """Fig. 1 labels: 0 rest, 1 E, 2 NE, 3 N, 4 NW, 5 W, 6 SW, 7 S, 8 SE."""
    c, _ = O.lattice(9)
    expect = [(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    assert [tuple(v[:2]) for v in c] == expect


def test_d3q19_groups_match_paper():
    """Eq. xi_i: i=0 rest, i=1-6 axis velocities (w=1/18), i=7-18 face diagonals (w=1/36)."""
    c, w = O.lattice(19)
    n2 = (c * c).sum(1)
    assert n2[0] == 0 and (n2[1:7] == 1).all() and (n2[7:] == 2).all()
    assert abs(w[0] - 1 / 3) < 1e-16 and np.allclose(w[1:7], 1 / 18) and np.allclose(w[7:], 1 / 36)


@pytest.mark.parametrize("q", LATTICES)
def test_equilibrium_moments(q):
    """Eqs. (fEq_herm), (moment_rho), (moment_rhoU): sum f0 = rho, sum c f0 = rho u,
    sum c c f0 = rho u u + rho c_s^2 I (Maxwellian second moment) to round-off."""
    rng = np.random.default_rng(1)
    c, _ = O.lattice(q)
    D = _D(q)
    for _ in range(20):
        rho, u = _rand_state(rng, q, 0.3)
        f = O.feq(q, rho, u)
        assert abs(f.sum() - rho) < 2e-15
        assert np.allclose(f @ c[:, :D], rho * u[:D], atol=2e-16, rtol=0)
        M2 = np.einsum("i,ia,ib->ab", f, c[:, :D], c[:, :D])
        assert np.allclose(M2, rho * np.outer(u[:D], u[:D]) + rho * CS2 * np.eye(D), atol=1e-15, rtol=0)


@pytest.mark.parametrize("q", LATTICES)
def test_third_moment_deviation_is_minus_Psi(q):
    """App. A: Psi is the deviation between the Maxwellian third moments and the
    ones of the truncated equilibrium; all 10 (D3Q19) / 4 (D2Q9) components are
    checked against the Maxwellian rho u u u + rho c_s^2 (u d + ...)."""
    rng = np.random.default_rng(2)
    c, _ = O.lattice(q)
    D = _D(q)
    for _ in range(10):
        rho, u = _rand_state(rng, q, 0.3)
        f = O.feq(q, rho, u)
        P = O.Psi_tensor(q, rho, u)
        for a, b, g in itertools.combinations_with_replacement(range(D), 3):
            lat = np.sum(c[:, a] * c[:, b] * c[:, g] * f)
            mx = rho * u[a] * u[b] * u[g] + rho * CS2 * (u[a] * (b == g) + u[b] * (a == g) + u[g] * (a == b))
            assert abs((lat - mx) + P[a, b, g]) < 1e-16, (a, b, g)
        # Psi is fully symmetric
        for a, b, g in itertools.permutations(range(3), 3):
            assert P[a, b, g] == P[g, a, b]


@pytest.mark.parametrize("q", LATTICES)
@pytest.mark.parametrize("s", [1, -1])
def test_psi_moments(q, s):
    """App. A Eq. (psi): psi carries no mass or momentum and its second Hermite
    moment is s * C (the full symmetric contraction counts off-diagonals twice)."""
    rng = np.random.default_rng(3)
    c, _ = O.lattice(q)
    D = _D(q)
    for _ in range(10):
        C6 = rng.normal(size=6)
        if D == 2:
            C6[[2, 4, 5]] = 0.0
        psi = O.psi(q, C6, s)
        assert abs(psi.sum()) < 1e-15
        assert np.allclose(psi @ c, 0.0, atol=1e-15)
        H2 = np.einsum("ia,ib->iab", c[:, :D], c[:, :D]) - CS2 * np.eye(D)
        M = np.einsum("iab,i->ab", H2, psi)
        Cm = np.zeros((3, 3))
        for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
            Cm[a, b] = Cm[b, a] = C6[k]
        assert np.allclose(M, s * Cm[:D, :D], atol=1e-14)


@pytest.mark.parametrize("q", LATTICES)
@pytest.mark.parametrize("sigma", [0.0, 0.98, 1.0])
def test_collision_conserves_mass_momentum(q, sigma):
    """Eq. (LBMscheme_reg): the regularised collision conserves rho and rho u to round-off
    for arbitrary populations, gradients, tau and sigma."""
    rng = np.random.default_rng(4)
    c, _ = O.lattice(q)
    for _ in range(30):
        rho, u = _rand_state(rng, q)
        f = O.feq(q, rho, u) * (1.0 + 0.05 * rng.normal(size=q))
        rho = f.sum()
        u = np.zeros(3)
        u[: _D(q)] = (f @ c[:, : _D(q)]) / rho
        S6 = 0.01 * rng.normal(size=6)
        C6 = 0.001 * rng.normal(size=6)
        tau = rng.uniform(0.5 + 1e-6, 2.0)
        fp = O.collide(q, f, rho, u, S6, C6, tau, sigma, -1)
        assert abs(fp.sum() - rho) < 1e-15 * 4
        assert np.allclose(fp @ c, f @ c, atol=4e-16)


@pytest.mark.parametrize("q", LATTICES)
def test_collision_tau_one_is_equilibrium(q):
    """tau = 1 removes the off-equilibrium part: f_post = f0 + psi/2; with C = 0, f_post = f0."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        rho, u = _rand_state(rng, q)
        f = O.feq(q, rho, u) + 1e-3 * rng.normal(size=q)
        fp = O.collide(q, f, rho, u, 0.01 * rng.normal(size=6), np.zeros(6), 1.0, 0.98, -1)
        assert np.allclose(fp, O.feq(q, rho, u), atol=1e-16)
        C6 = 1e-3 * rng.normal(size=6)
        fp = O.collide(q, f, rho, u, np.zeros(6), C6, 1.0, 0.5, -1)
        assert np.allclose(fp, O.feq(q, rho, u) + 0.5 * O.psi(q, C6, -1), atol=1e-16)


@pytest.mark.parametrize("q", LATTICES)
def test_projection_recovers_hermite_coefficient(q):
    """Eq. (a1Proj) with sigma = 1 and psi = 0 projects f - f0 on H2: for
    f = f0 + w_i H2_i:A/(2 c_s^4) + (a component orthogonal to H2) it returns A.
    With sigma = 0 it returns the finite-difference value -2 tau rho c_s^2 S."""
    rng = np.random.default_rng(6)
    c, w = O.lattice(q)
    D = _D(q)
    H2 = np.einsum("ia,ib->iab", c[:, :D], c[:, :D]) - CS2 * np.eye(D)
    for _ in range(5):
        rho, u = _rand_state(rng, q)
        A = rng.normal(size=(D, D)) * 1e-3
        A = A + A.T
        f1 = w * np.einsum("iab,ab->i", H2, A) / (2 * CS2 * CS2)
        f = O.feq(q, rho, u) + f1
        a1 = O.a1(q, f, rho, u, np.zeros(6), np.zeros(6), 0.7, 1.0, -1)
        idx = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        for k, (a, b) in enumerate(idx):
            if a < D and b < D:
                assert abs(a1[k] - A[a, b]) < 1e-16
        S6 = rng.normal(size=6) * 1e-2
        a1 = O.a1(q, f, rho, u, S6, np.zeros(6), 0.7, 0.0, -1)
        for k, (a, b) in enumerate(idx):
            if a < D and b < D:
                assert abs(a1[k] - (-2 * 0.7 * rho * CS2 * S6[k])) < 1e-16


def test_regularised_offequilibrium_moments_d2q9():
    """Eqs. (fNEq_herm), (a13RR) on D2Q9 (whose H3_xxy, H3_xyy are orthogonal):
    the regularised f1 has zeroth and first moments 0, second Hermite moment a1
    and third Hermite moments a1_aab = 2 u_a a1_ab + u_b a1_aa."""
    q, D = 9, 2
    rng = np.random.default_rng(7)
    c, w = O.lattice(q)
    tau = 2.0
    for _ in range(10):
        rho, u = _rand_state(rng, q, 0.3)
        f = O.feq(q, rho, u) * (1 + 0.02 * rng.normal(size=q))
        rho = f.sum()
        u = np.zeros(3)
        u[:D] = f @ c[:, :D] / rho
        fp = O.collide(q, f, rho, u, np.zeros(6), np.zeros(6), tau, 1.0, -1)
        f1 = (fp - O.feq(q, rho, u)) / (1.0 - 1.0 / tau)
        a1v = O.a1(q, f, rho, u, np.zeros(6), np.zeros(6), tau, 1.0, -1)
        A = np.array([[a1v[0], a1v[3]], [a1v[3], a1v[1]]])
        assert abs(f1.sum()) < 1e-16 and np.allclose(f1 @ c[:, :D], 0, atol=1e-16)
        H2 = np.einsum("ia,ib->iab", c[:, :D], c[:, :D]) - CS2 * np.eye(D)
        assert np.allclose(np.einsum("iab,i->ab", H2, f1), A, atol=1e-16)
        for a, b in [(0, 1), (1, 0)]:
            H3 = (c[:, a] ** 2 - CS2) * c[:, b]
            assert abs(H3 @ f1 - (2 * u[a] * A[a, b] + u[b] * A[a, a])) < 1e-16


def _acoustic_decay_rate(mach, s, nx=64, steps=200):
    d = {"lattice": 9, "coarse_n": (nx, 4), "boxes": [], "nu0": 0.1, "sigma": 1.0, "dc_variant": 2, "psi_sign": s}
    h = O.Hierarchy(d)
    x = np.tile(np.arange(nx), 4).astype(float)
    k = 2 * np.pi / nx
    A, U = 1e-4, mach * math.sqrt(CS2)
    h.init(0, 1 + A * np.cos(k * x), np.stack([U + A * math.sqrt(CS2) * np.cos(k * x), 0 * x]))
    amps = []
    for _ in range(steps // 20):
        r, _ = h.macros(0)
        amps.append(abs(np.fft.fft(r[:nx])[1]))
        h.advance(20)
    ts = np.arange(len(amps)) * 20
    return -np.polyfit(ts, np.log(amps), 1)[0], k


def test_psi_sign_restores_galilean_invariance():
    """Reading R1 (App. A, Eq. psi): the cubic-Mach correction exists to remove
    the U-dependent error of the rho u^3 moment.  A travelling acoustic wave
    along a mean flow U_x must decay at the same rate for every U (isothermal
    linear theory: Gamma = nu k^2 for D2Q9 with sigma = 1).  The sign -1 on psi
    (with Psi as printed) achieves this; the printed +1 doubles the defect."""
    rates_m = [_acoustic_decay_rate(m, -1)[0] for m in (0.0, 0.2, 0.4)]
    rates_p = [_acoustic_decay_rate(m, +1)[0] for m in (0.0, 0.2, 0.4)]
    k = 2 * np.pi / 64
    assert max(abs(r - rates_m[0]) for r in rates_m) < 0.005 * rates_m[0]
    assert abs(rates_m[0] - 0.1 * k * k) < 0.03 * 0.1 * k * k
    assert rates_p[2] < 0.7 * rates_p[0]  # the opposite sign visibly breaks invariance
