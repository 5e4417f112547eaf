"""Seeded synthetic workloads: hierarchy descriptions and initial fields.

This module holds no arithmetic of the lattice Boltzmann method itself; it
only describes the geometry of each workload and evaluates the analytic
initial fields (density and velocity) at every node of every level.  The
CUDA library and the CPU oracle both receive these arrays.

Workloads (all lattice units; positions in level-0 node units; Mach numbers
relative to c_s = 1/sqrt(3)):

* ``vortex2d_2lvl``   D2Q9, 128^2 periodic, one patch of 64^2 coarse cells,
  barotropic vortex (paper Sec. 4.2, Eq. init_COVO) of core radius 8, max swirl
  Mach 0.05, carried diagonally at Mach 0.1 across the interface, 200 steps.
* ``pulse2d_3lvl``    D2Q9, 512^2 periodic, nested patches of 256^2 and 128^2
  coarse cells, Gaussian density pulse (paper Sec. 4.1, Eq. init_Pulse, radial
  form) of amplitude 1e-3 and half-width 6 finest cells in a Mach-0.2 mean
  flow along x, 2000 steps.
* ``vortex3d_3lvl``   D3Q19, 256^3 periodic, nested cubes of 128^3 and 64^3
  coarse cells, vortex tube along z plus 1 % white noise at Mach 0.1, 500 steps.
* ``slab3d_3lvl``     D3Q19, 512x512x256, a level-1 slab spanning x and y
  (z in [96,160)) and a level-2 box, pulse 1e-4 plus vortex at Mach 0.15, 300 steps.
* ``batch2d``         96 independent 2-level D2Q9 hierarchies of seeded sizes.

Every random draw comes from numpy's PCG64 seeded by the workload seed, or,
for white noise, from SplitMix64 keyed by (seed, finest-level integer
coordinates) so that co-located nodes of different levels agree bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

CS = 1.0 / math.sqrt(3.0)


# ----------------------------------------------------------------- geometry
def level_geometry(desc: dict, l: int):
    """(n[3], off[3], periodic[3]) of level l: level 0 is the periodic coarse
    box; a patch [lo,hi) in level-0 cells has (hi-lo)*2^l+1 nodes per axis
    (cell-vertex, shared interface nodes) unless it spans a periodic axis."""
    D = 2 if desc["lattice"] == 9 else 3
    cn = list(desc["coarse_n"]) + [1] * (3 - len(desc["coarse_n"]))
    n, off, per = [1, 1, 1], [0, 0, 0], [1, 1, 1]
    for a in range(D):
        if l == 0:
            n[a], off[a], per[a] = cn[a], 0, 1
            continue
        lo, hi = desc["boxes"][l - 1][0][a], desc["boxes"][l - 1][1][a]
        if lo == 0 and hi == cn[a]:
            n[a], off[a], per[a] = cn[a] << l, 0, 1
        else:
            n[a], off[a], per[a] = ((hi - lo) << l) + 1, lo << l, 0
    return tuple(n), tuple(off), tuple(per)


def n_levels(desc: dict) -> int:
    return 1 + len(desc.get("boxes", []))


def level_axes(desc: dict, l: int):
    """Node positions of level l in level-0 units along each axis, shaped to broadcast
    to (nz, ny, nx): x (1, 1, nx), y (1, ny, 1), z (nz, 1, 1)."""
    n, off, _ = level_geometry(desc, l)
    s = 1.0 / (1 << l)
    return ((np.arange(n[0]) + off[0]) * s).reshape(1, 1, -1), ((np.arange(n[1]) + off[1]) * s).reshape(1, -1, 1), \
        ((np.arange(n[2]) + off[2]) * s).reshape(-1, 1, 1)


def level_positions(desc: dict, l: int):
    """Node positions of level l in level-0 units, arrays of shape (nz, ny, nx)."""
    n, _, _ = level_geometry(desc, l)
    shape = (n[2], n[1], n[0])
    return tuple(np.broadcast_to(a, shape).copy() for a in level_axes(desc, l))


def level_int_coords(desc: dict, l: int):
    """Integer coordinates of level-l nodes on the finest level's lattice."""
    n, off, _ = level_geometry(desc, l)
    L = n_levels(desc) - 1
    sh = L - l
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return ((x + off[0]) << sh, (y + off[1]) << sh, (z + off[2]) << sh)


def node_counts(desc: dict):
    """Active node count of every level (the level box minus the nodes strictly
    inside the next level's patch)."""
    out = []
    L = n_levels(desc)
    for l in range(L):
        n, off, per = level_geometry(desc, l)
        tot = n[0] * n[1] * n[2]
        if l + 1 < L:
            nc, offc, perc = level_geometry(desc, l + 1)
            hole = 1
            for a in range(3):
                if nc[a] == 1 and n[a] == 1:
                    continue
                if perc[a]:
                    hole *= n[a]
                else:
                    hole *= ((nc[a] - 1) >> 1) - 1
            tot -= hole
        out.append(tot)
    return out


def updates_per_coarse_step(desc: dict) -> int:
    return sum(c << l for l, c in enumerate(node_counts(desc)))


def fine_equivalent_per_coarse_step(desc: dict) -> int:
    """Node updates of a uniform finest-level grid over the whole domain."""
    L = n_levels(desc) - 1
    D = 2 if desc["lattice"] == 9 else 3
    cn = list(desc["coarse_n"]) + [1] * (3 - len(desc["coarse_n"]))
    tot = 1
    for a in range(D):
        tot *= cn[a] << L
    return tot << L


# ---------------------------------------------------------------- fields
def _min_image(d, period):
    return d - period * np.round(d / period)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def hashed_normal(seed: int, stream: int, ix, iy, iz) -> np.ndarray:
    """Standard normal keyed by (seed, stream, integer coordinates), Box-Muller."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(0x100000001B3) + np.uint64(stream)).astype(np.uint64)
        k = splitmix64(key ^ splitmix64(ix.astype(np.uint64)
                                        ^ splitmix64(iy.astype(np.uint64) * np.uint64(3)
                                                     ^ splitmix64(iz.astype(np.uint64) * np.uint64(7)))))
        a = splitmix64(k)
        b = splitmix64(k ^ np.uint64(0xD1B54A32D192ED03))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    u2 = ((b >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def vortex_fields(x, y, xc, yc, Rc, swirl_mach, U, period=None):
    """Barotropic vortex (Eq. init_COVO) carried by the mean flow U=(Ux,Uy[,Uz]).
    eps is chosen so that the maximum swirl speed eps*exp(-1/2) equals
    swirl_mach * c_s."""
    eps = swirl_mach * CS * math.exp(0.5)
    dx, dy = x - xc, y - yc
    if period is not None:
        dx, dy = _min_image(dx, period[0]), _min_image(dy, period[1])
    r2 = (dx * dx + dy * dy) / (Rc * Rc)
    rho = np.exp(-(eps * eps) / (2.0 * CS * CS) * np.exp(-r2))
    g = eps * np.exp(-0.5 * r2) / Rc
    ux = U[0] - g * dy
    uy = U[1] + g * dx
    uz = np.full_like(x, U[2] if len(U) > 2 else 0.0)
    return rho, ux, uy, uz


def pulse_fields(x, y, z, xc, yc, zc, Rc, A, U, period=None, dims=2):
    """Gaussian density pulse rho = 1 + A exp(-r^2/(2 Rc^2)) (Eq. init_Pulse,
    radial form) in the uniform mean flow U."""
    dx, dy, dz = x - xc, y - yc, (z - zc) if dims == 3 else 0.0 * z
    if period is not None:
        dx, dy = _min_image(dx, period[0]), _min_image(dy, period[1])
        if dims == 3:
            dz = _min_image(dz, period[2])
    r2 = dx * dx + dy * dy + (dz * dz if dims == 3 else 0.0)
    rho = 1.0 + A * np.exp(-r2 / (2.0 * Rc * Rc))
    return rho, np.full_like(x, U[0]), np.full_like(x, U[1]), np.full_like(x, U[2] if len(U) > 2 else 0.0)


# ---------------------------------------------------------------- workloads
def _base(lattice, coarse_n, boxes, nu0=1e-5, storage="f64"):
    return {"lattice": lattice, "coarse_n": tuple(coarse_n), "boxes": [tuple(map(tuple, b)) for b in boxes],
            "nu0": nu0, "sigma": 0.98, "dc_variant": 2, "psi_sign": -1, "storage": storage}


def vortex2d(n=128, patch=(32, 96), steps=200, seed=0, storage="f64", nu0=1e-5, swirl=0.05, mach=0.1,
             Rc=8.0, centre=None, levels=2):
    """2-D vortex crossing a plane refinement interface (paper Sec. 4.2 analogue)."""
    boxes = [((patch[0], patch[0]), (patch[1], patch[1]))]
    if levels == 3:
        q = (patch[1] - patch[0]) // 4
        boxes.append(((patch[0] + q, patch[0] + q), (patch[1] - q, patch[1] - q)))
    d = _base(9, (n, n), boxes, nu0, storage)
    rng = np.random.default_rng(seed)
    c = centre if centre is not None else (patch[1] - n / 16.0, 0.5 * n)
    jit = rng.uniform(-2.0, 2.0, 2)
    U = mach * CS
    d["init"] = {"kind": "vortex", "xc": c[0] + jit[0], "yc": c[1] + jit[1], "Rc": Rc, "swirl": swirl,
                 "U": (U / math.sqrt(2.0), U / math.sqrt(2.0), 0.0)}
    d["steps"] = steps
    d["name"] = f"vortex2d_{levels}lvl_{n}"
    return d


def pulse2d(n=512, boxes=((128, 384), (192, 320)), steps=2000, seed=0, storage="f64", nu0=1e-5,
            A=1e-3, Rc_finest=6.0, mach=0.2):
    """2-D acoustic pulse radiating across two nested interfaces (paper Sec. 4.1 analogue)."""
    bx = [((lo, lo), (hi, hi)) for lo, hi in boxes]
    d = _base(9, (n, n), bx, nu0, storage)
    rng = np.random.default_rng(seed)
    L = len(boxes)
    jit = rng.uniform(-16.0 * n / 512, 16.0 * n / 512, 2)
    d["init"] = {"kind": "pulse", "xc": 0.5 * n + jit[0], "yc": 0.5 * n + jit[1], "zc": 0.0,
                 "Rc": Rc_finest / (1 << L), "A": A, "U": (mach * CS, 0.0, 0.0)}
    d["steps"] = steps
    d["name"] = f"pulse2d_{L + 1}lvl_{n}"
    return d


def vortex3d(n=256, boxes=((64, 192), (96, 160)), steps=500, seed=0, storage="f32", nu0=1e-5,
             swirl=0.05, mach=0.1, Rc=8.0, noise=0.01):
    """3-D vortex tube along z with seeded white noise (D3Q19, nested cubes)."""
    bx = [((lo, lo, lo), (hi, hi, hi)) for lo, hi in boxes]
    d = _base(19, (n, n, n), bx, nu0, storage)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-2.0, 2.0, 2)
    d["init"] = {"kind": "vortex", "xc": 0.5 * n + jit[0], "yc": 0.5 * n + jit[1], "Rc": Rc * n / 256,
                 "swirl": swirl, "U": (mach * CS, 0.0, 0.0), "noise": noise, "seed": seed}
    d["steps"] = steps
    d["name"] = f"vortex3d_{len(boxes) + 1}lvl_{n}"
    return d


def slab3d(nxy=512, nz=256, slab=(96, 160), box=((128, 128, 112), (384, 384, 144)), steps=300, seed=0,
           storage="f16s", nu0=1e-5, mach=0.15, A=1e-4):
    """3-D slab refinement spanning x and y with an inner refined box."""
    bx = [((0, 0, slab[0]), (nxy, nxy, slab[1])), box]
    d = _base(19, (nxy, nxy, nz), bx, nu0, storage)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-2.0, 2.0, 3)
    zc = 0.5 * (box[0][2] + box[1][2])
    d["init"] = {"kind": "pulse+vortex", "xc": 0.5 * nxy + jit[0], "yc": 0.5 * nxy + jit[1], "zc": zc + jit[2],
                 "Rc": 8.0 * nxy / 512, "A": A, "swirl": 0.05, "U": (mach * CS, 0.0, 0.0)}
    d["steps"] = steps
    d["name"] = f"slab3d_{nxy}x{nxy}x{nz}"
    return d


def circle_mask(box, centre, radius):
    """Staircase refinement region (paper Sec. 4.1.2): the level-0 cells of the box
    ((lo_x, lo_y), (hi_x, hi_y)) whose centre lies inside the circle; uint8 array of
    shape (ny, nx) over the box's cells, x fastest."""
    (lx, ly), (hx, hy) = box
    y, x = np.meshgrid(np.arange(ly, hy) + 0.5, np.arange(lx, hx) + 0.5, indexing="ij")
    return ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 < radius * radius).astype(np.uint8)


def inclined_mask(box, point, angle_deg):
    """Staircase refinement region (paper Sec. 4.2.2): the level-0 cells of the box whose
    centre lies below the line through `point` inclined by angle_deg to the x axis."""
    (lx, ly), (hx, hy) = box
    y, x = np.meshgrid(np.arange(ly, hy) + 0.5, np.arange(lx, hx) + 0.5, indexing="ij")
    t = math.tan(math.radians(angle_deg))
    return (y < point[1] + t * (x - point[0])).astype(np.uint8)


def pulse_circle(n=64, box=((12, 12), (52, 52)), radius=16.0, steps=60, seed=0, storage="f64", nu0=1e-5, A=1e-3,
                 Rc_fine=3.0, mach=0.0):
    """2-D acoustic pulse inside a circular refined region (paper Sec. 4.1.2 analogue):
    D2Q9, two levels, the refined cells those of the box within `radius` of the
    domain centre; the pulse starts at the centre (seeded jitter) and radiates across
    the staircase interface."""
    d = _base(9, (n, n), [box], nu0, storage)
    c = (0.5 * n, 0.5 * n)
    d["masks"] = [None, circle_mask(box, c, radius)]
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-1.0, 1.0, 2)
    d["init"] = {"kind": "pulse", "xc": c[0] + jit[0], "yc": c[1] + jit[1], "zc": 0.0, "Rc": Rc_fine / 2.0, "A": A,
                 "U": (mach * CS, 0.0, 0.0)}
    d["steps"] = steps
    d["name"] = f"pulse_circle_{n}"
    return d


def vortex_inclined(n=64, box=((8, 8), (56, 56)), angle=30.0, steps=60, seed=0, storage="f64", nu0=1e-5, swirl=0.05,
                    mach=0.1, Rc=4.0):
    """2-D vortex convected across a 30-degree inclined staircase interface (paper Sec.
    4.2.2 analogue): D2Q9, two levels, the refined cells those of the box below the
    line through the domain centre at `angle`; the vortex starts below the line and
    the mean flow carries it across, normal to the line."""
    d = _base(9, (n, n), [box], nu0, storage)
    c = (0.5 * n, 0.5 * n)
    d["masks"] = [None, inclined_mask(box, c, angle)]
    a = math.radians(angle)
    nrm = (-math.sin(a), math.cos(a))  # unit normal pointing to the coarse side
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-1.0, 1.0, 2)
    U = mach * CS
    d["init"] = {"kind": "vortex", "xc": c[0] - 2.0 * Rc * nrm[0] + jit[0], "yc": c[1] - 2.0 * Rc * nrm[1] + jit[1],
                 "Rc": Rc, "swirl": swirl, "U": (U * nrm[0], U * nrm[1], 0.0)}
    d["steps"] = steps
    d["name"] = f"vortex_inclined_{n}"
    return d


def init_fields(desc: dict, l: int):
    """(rho, u) of every node of level l, rho shape (N,), u shape (D, N)."""
    D = 2 if desc["lattice"] == 9 else 3
    # per-axis positions: every field below is evaluated by broadcasting (the same
    # per-node arithmetic as on full coordinate arrays) and expanded to the level's
    # box at the end
    x, y, z = level_axes(desc, l)
    n, _, _ = level_geometry(desc, l)
    shape = (n[2], n[1], n[0])
    ini = desc["init"]
    cn = list(desc["coarse_n"]) + [1] * (3 - len(desc["coarse_n"]))
    per = (float(cn[0]), float(cn[1]), float(cn[2]))
    if ini["kind"] == "vortex":
        rho, ux, uy, uz = vortex_fields(x, y, ini["xc"], ini["yc"], ini["Rc"], ini["swirl"], ini["U"], per)
    elif ini["kind"] == "pulse":
        rho, ux, uy, uz = pulse_fields(x, y, z, ini["xc"], ini["yc"], ini.get("zc", 0.0), ini["Rc"], ini["A"],
                                       ini["U"], per, dims=D)
    elif ini["kind"] == "pulse+vortex":
        rho_p, _, _, _ = pulse_fields(x, y, z, ini["xc"], ini["yc"], ini["zc"], ini["Rc"], ini["A"], (0, 0, 0),
                                      per, dims=D)
        rho_v, ux, uy, uz = vortex_fields(x, y, ini["xc"] - 4 * ini["Rc"], ini["yc"], ini["Rc"], ini["swirl"],
                                          ini["U"], per)
        rho = rho_v * rho_p
    elif ini["kind"] == "uniform":
        rho = np.full(shape, ini.get("rho", 1.0))
        U = ini["U"]
        ux, uy, uz = np.full(shape, U[0]), np.full(shape, U[1]), np.full(shape, U[2] if len(U) > 2 else 0.0)
    else:
        raise ValueError(ini["kind"])
    rho, ux, uy, uz = (np.broadcast_to(np.asarray(a, dtype=np.float64), shape) for a in (rho, ux, uy, uz))
    if ini.get("noise", 0.0) > 0.0:
        ix, iy, iz = level_int_coords(desc, l)
        amp = ini["noise"] * math.sqrt(sum(v * v for v in ini["U"]))
        ux = ux + amp * hashed_normal(ini.get("seed", 0), 1, ix, iy, iz)
        uy = uy + amp * hashed_normal(ini.get("seed", 0), 2, ix, iy, iz)
        if D == 3:
            uz = uz + amp * hashed_normal(ini.get("seed", 0), 3, ix, iy, iz)
    u = np.empty((D,) + shape)
    for a, v in enumerate([ux, uy, uz][:D]):
        u[a] = v
    return np.ascontiguousarray(rho).reshape(-1), u.reshape(D, -1)


def batch2d(n=96, steps=1000, seed=0, storage="f32", nu0=1e-5, sides=(96, 128, 192, 256, 384, 512, 768, 1024)):
    """Independent 2-level D2Q9 hierarchies of seeded uneven sizes: coarse side drawn
    uniformly from `sides`, a centred patch of half the side; each carries a seeded
    barotropic vortex (swirl Mach U[0.02, 0.08], mean Mach U[0.05, 0.15], random
    direction) or an acoustic pulse (amplitude log-uniform in [1e-4, 1e-3])."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice(sides))
        lo, hi = side // 4, 3 * side // 4
        d = _base(9, (side, side), [((lo, lo), (hi, hi))], nu0, storage)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        if rng.random() < 0.5:
            mach = rng.uniform(0.05, 0.15) * CS
            d["init"] = {"kind": "vortex", "xc": 0.5 * side + rng.uniform(-2, 2), "yc": 0.5 * side + rng.uniform(-2, 2),
                         "Rc": side / 16.0, "swirl": float(rng.uniform(0.02, 0.08)),
                         "U": (mach * math.cos(ang), mach * math.sin(ang), 0.0)}
        else:
            d["init"] = {"kind": "pulse", "xc": 0.5 * side + rng.uniform(-2, 2), "yc": 0.5 * side + rng.uniform(-2, 2),
                         "zc": 0.0, "Rc": side / 64.0, "A": float(10.0 ** rng.uniform(-4.0, -3.0)),
                         "U": (0.1 * CS * math.cos(ang), 0.1 * CS * math.sin(ang), 0.0)}
        d["steps"] = steps
        d["name"] = f"batch2d_{k}_{side}"
        out.append(d)
    return out


CONFIGS = {
    "vortex2d_2lvl": lambda **kw: vortex2d(**kw),
    "pulse2d_3lvl": lambda **kw: pulse2d(**kw),
    "vortex3d_3lvl": lambda **kw: vortex3d(**kw),
    "slab3d_3lvl": lambda **kw: slab3d(**kw),
}
