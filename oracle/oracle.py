"""ctypes view of the FP64 CPU oracle (oracle/dc_lbm_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the checker of the CUDA library of
this repository; only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path and never imports it.

The shared library is built by ``build()`` (plain gcc, no CUDA).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_oracle.so")
# the same source built with -fopenmp: the per-node loops of a step are shared out
# over threads, every node's arithmetic is unchanged (identical bits)
LIB_OMP_PATH = os.path.join(HERE, "liblbm_oracle_omp.so")
SRC = os.path.join(HERE, "dc_lbm_oracle.c")

HOLE, BULK, TFP, IE, TFC = 0, 1, 2, 3, 4
MAX_LEVELS = 4


def _gcc(out, extra):
    src_t = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "dc_lbm_oracle.h")))
    if not os.path.exists(out) or os.path.getmtime(out) < src_t:
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", *extra,
                               "-o", out, SRC, "-lm"])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single translation unit, -O2, no -ffast-math, no
    contraction), once plain and once with -fopenmp."""
    if force:
        for p in (LIB_PATH, LIB_OMP_PATH):
            if os.path.exists(p):
                os.remove(p)
    _gcc(LIB_PATH, [])
    _gcc(LIB_OMP_PATH, ["-fopenmp"])
    return LIB_PATH


class _Desc(C.Structure):
    _fields_ = [
        ("lattice", C.c_int),
        ("n_levels", C.c_int),
        ("coarse_n", C.c_long * 3),
        ("box_lo", (C.c_long * 3) * MAX_LEVELS),
        ("box_hi", (C.c_long * 3) * MAX_LEVELS),
        ("nu0", C.c_double),
        ("sigma", C.c_double),
        ("dc_variant", C.c_int),
        ("psi_sign", C.c_int),
        ("mask", C.c_void_p * MAX_LEVELS),
    ]


_libs = {}


def lib(threaded: bool = False):
    """The plain build, or with threaded=True the OpenMP build."""
    if threaded not in _libs:
        build()
        L = C.CDLL(LIB_OMP_PATH if threaded else LIB_PATH)
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Desc), C.c_char_p, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_level_info.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_long), C.POINTER(C.c_long),
                                     C.POINTER(C.c_int), dp]
        L.orc_node_class.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.orc_known_masks.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.orc_init.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_advance.argtypes = [C.c_void_p, C.c_long]
        L.orc_get_macros.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_get_pops.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_pops.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_gradients.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_max_newton_iters.argtypes = [C.c_void_p]
        L.orc_node_updates.argtypes = [C.c_void_p]
        L.orc_node_updates.restype = C.c_long
        L.orc_error.argtypes = [C.c_void_p]
        L.orc_error.restype = C.c_char_p
        L.orc_lattice.argtypes = [C.c_int, C.c_void_p, dp]
        L.orc_feq.argtypes = [C.c_int, C.c_double, dp, dp]
        L.orc_psi.argtypes = [C.c_int, dp, C.c_int, dp]
        L.orc_Psi_tensor.argtypes = [C.c_int, C.c_double, dp, dp]
        L.orc_collide.argtypes = [C.c_int, dp, C.c_double, dp, dp, dp, C.c_double, C.c_double,
                                  C.c_int, dp]
        L.orc_a1.argtypes = [C.c_int, dp, C.c_double, dp, dp, dp, C.c_double, C.c_double, C.c_int, dp]
        L.orc_newton_system.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.orc_newton.argtypes = [C.c_int, dp, dp, dp]
        L.orc_tempint_weights.argtypes = [dp]
        L.orc_lagrange4_weights.argtypes = [C.c_int, dp]
        L.orc_known_from_occupancy.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_threads.argtypes = [C.c_int]
        L.orc_ie_stencil.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_void_p, dp]
        _libs[threaded] = L
    return _libs[threaded]


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build's node loops: sets the count when n > 0; returns it."""
    return lib(True).orc_threads(int(n))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size < n:
        a = np.concatenate([a.ravel(), np.zeros(n - a.size)])
    return a


# ---------------------------------------------------------------- node-local
def lattice(q: int):
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    r = lib().orc_lattice(q, c.ctypes.data_as(C.c_void_p), _dp(w))
    if r < 0:
        raise ValueError("lattice must be 9 or 19")
    return c, w


def feq(q, rho, u):
    out = np.zeros(q)
    lib().orc_feq(q, float(rho), _dp(_f64(u, 3)), _dp(out))
    return out


def psi(q, C6, psi_sign):
    out = np.zeros(q)
    lib().orc_psi(q, _dp(_f64(C6, 6)), int(psi_sign), _dp(out))
    return out


def Psi_tensor(q, rho, u):
    out = np.zeros(27)
    lib().orc_Psi_tensor(q, float(rho), _dp(_f64(u, 3)), _dp(out))
    return out.reshape(3, 3, 3)


def collide(q, f, rho, u, S6, C6, tau, sigma, psi_sign):
    out = np.zeros(q)
    lib().orc_collide(q, _dp(_f64(f)), float(rho), _dp(_f64(u, 3)), _dp(_f64(S6, 6)),
                      _dp(_f64(C6, 6)), float(tau), float(sigma), int(psi_sign), _dp(out))
    return out


def a1(q, f, rho, u, S6, C6, tau, sigma, psi_sign):
    out = np.zeros(6)
    lib().orc_a1(q, _dp(_f64(f)), float(rho), _dp(_f64(u, 3)), _dp(_f64(S6, 6)), _dp(_f64(C6, 6)),
                 float(tau), float(sigma), int(psi_sign), _dp(out))
    return out


def newton_system(q, fhat, gamma, X):
    n = 3 if q == 9 else 4
    F = np.zeros(n)
    J = np.zeros(n * n)
    lib().orc_newton_system(q, _dp(_f64(fhat)), _dp(_f64(gamma)), _dp(_f64(X, 4)), _dp(F), _dp(J))
    return F, J.reshape(n, n)


def newton(q, fhat, gamma):
    X = np.zeros(4)
    it = lib().orc_newton(q, _dp(_f64(fhat)), _dp(_f64(gamma)), _dp(X))
    return X[: (3 if q == 9 else 4)], it


def tempint_weights():
    w = np.zeros(3)
    lib().orc_tempint_weights(_dp(w))
    return w


def lagrange4_weights(one_sided: bool):
    w = np.zeros(4)
    lib().orc_lagrange4_weights(int(one_sided), _dp(w))
    return w


def known_from_occupancy(q, occ_f, occ_c):
    """Set rule on 3x3(x3) occupancy grids indexed [oz+1][oy+1][ox+1]; returns (kf, kc) bit masks."""
    of = np.ascontiguousarray(np.asarray(occ_f, dtype=np.uint8).reshape(-1))
    oc = np.ascontiguousarray(np.asarray(occ_c, dtype=np.uint8).reshape(-1))
    if of.size == 9:
        of = np.concatenate([np.zeros(9, np.uint8), of, np.zeros(9, np.uint8)])
        oc = np.concatenate([np.zeros(9, np.uint8), oc, np.zeros(9, np.uint8)])
    kf = C.c_uint()
    kc = C.c_uint()
    lib().orc_known_from_occupancy(q, of.ctypes.data_as(C.c_void_p), oc.ctypes.data_as(C.c_void_p),
                                   C.byref(kf), C.byref(kc))
    return kf.value, kc.value


# ---------------------------------------------------------------- hierarchy
class Hierarchy:
    """A multi-level DC hierarchy advanced by the oracle (Sec. 3.5).

    desc keys: lattice (9|19), coarse_n (nx, ny[, nz]), boxes [((lo),(hi)), ...]
    for levels 1.. in level-0 cell units, nu0, sigma, dc_variant, psi_sign, and
    optionally masks: per level None or a uint8 array over the parent cells of the
    level's box (shape (ny, nx) in 2-D, nonzero = refined; a staircase region).
    threaded=True runs the per-node loops of every step on the OpenMP build (same
    arithmetic per node, identical results).
    """

    def __init__(self, desc: dict, threaded: bool = False):
        self._L = lib(threaded)
        d = _Desc()
        d.lattice = int(desc["lattice"])
        boxes = desc.get("boxes", [])
        d.n_levels = 1 + len(boxes)
        cn = list(desc["coarse_n"]) + [1] * (3 - len(desc["coarse_n"]))
        for a in range(3):
            d.coarse_n[a] = int(cn[a])
        for l, (lo, hi) in enumerate(boxes, start=1):
            for a in range(3):
                d.box_lo[l][a] = int(lo[a]) if a < len(lo) else 0
                d.box_hi[l][a] = int(hi[a]) if a < len(hi) else 1
        d.nu0 = float(desc["nu0"])
        d.sigma = float(desc.get("sigma", 0.98))
        d.dc_variant = int(desc.get("dc_variant", 2))
        d.psi_sign = int(desc.get("psi_sign", -1))
        # staircase regions: masks[l] over the parent cells of level l's box (x fastest)
        self._masks = []
        for l, m in enumerate(desc.get("masks") or []):
            if m is None or l == 0:
                continue
            arr = np.ascontiguousarray(np.asarray(m, dtype=np.uint8))
            self._masks.append(arr)
            d.mask[l] = arr.ctypes.data
        err = C.create_string_buffer(256)
        self._h = self._L.orc_create(C.byref(d), err, 256)
        if not self._h:
            raise ValueError("oracle: " + err.value.decode())
        self.q = d.lattice
        self.D = 2 if self.q == 9 else 3
        self.n_levels = d.n_levels
        self.levels = [self.level_info(l) for l in range(self.n_levels)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def level_info(self, l):
        n = (C.c_long * 3)()
        off = (C.c_long * 3)()
        per = (C.c_int * 3)()
        tau = C.c_double()
        if self._L.orc_level_info(self._h, l, n, off, per, C.byref(tau)) != 0:
            raise IndexError(l)
        return {"n": tuple(n), "off": tuple(off), "periodic": tuple(per), "tau": tau.value,
                "N": n[0] * n[1] * n[2]}

    def node_class(self, l):
        N = self.levels[l]["N"]
        out = np.zeros(N, dtype=np.uint8)
        self._L.orc_node_class(self._h, l, out.ctypes.data_as(C.c_void_p))
        return out

    def known_masks(self, l):
        N = self.levels[l]["N"]
        kf = np.zeros(N, dtype=np.uint32)
        kc = np.zeros(N, dtype=np.uint32)
        self._L.orc_known_masks(self._h, l, kf.ctypes.data_as(C.c_void_p), kc.ctypes.data_as(C.c_void_p))
        return kf, kc

    def init(self, l, rho, u):
        N = self.levels[l]["N"]
        rho = _f64(rho).reshape(N)
        u3 = np.zeros((3, N))
        u = np.asarray(u, dtype=np.float64).reshape(-1, N)
        u3[: u.shape[0]] = u
        if self._L.orc_init(self._h, l, _dp(rho), _dp(np.ascontiguousarray(u3))) != 0:
            raise RuntimeError("orc_init failed")

    def advance(self, n):
        if self._L.orc_advance(self._h, int(n)) != 0:
            raise RuntimeError("oracle: " + self._L.orc_error(self._h).decode())

    def macros(self, l):
        N = self.levels[l]["N"]
        rho = np.zeros(N)
        u = np.zeros((self.D, N))
        self._L.orc_get_macros(self._h, l, _dp(rho), _dp(u))
        return rho, u

    def pops(self, l):
        N = self.levels[l]["N"]
        f = np.zeros((self.q, N))
        self._L.orc_get_pops(self._h, l, _dp(f))
        return f

    def gradients(self, l):
        """(S, C) last supplied to the interface nodes of level l, each [6, N]."""
        N = self.levels[l]["N"]
        S = np.zeros((6, N))
        Cm = np.zeros((6, N))
        if self._L.orc_get_gradients(self._h, l, _dp(S), _dp(Cm)) != 0:
            raise IndexError(l)
        return S, Cm

    def ie_stencil(self, l, idx):
        """(points [n, 3] in level-l coordinates, weights [n]) of hanging node idx."""
        pts = np.zeros((16, 3), dtype=np.int64)
        w = np.zeros(16)
        n = self._L.orc_ie_stencil(self._h, int(l), int(idx), pts.ctypes.data_as(C.c_void_p), _dp(w))
        if n < 0:
            raise ValueError(f"node {idx} of level {l} has no hanging-node stencil")
        return pts[:n], w[:n]

    def set_pops(self, l, f):
        f = _f64(f)
        self._L.orc_set_pops(self._h, l, _dp(f))

    @property
    def max_newton_iters(self):
        return self._L.orc_max_newton_iters(self._h)

    @property
    def node_updates(self):
        return self._L.orc_node_updates(self._h)
