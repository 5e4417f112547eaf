"""Thin ctypes binding of the C-ABI in ``include/lbm.h`` (same names, argument
marshalling only).  Every step of the method runs in the CUDA library
``_lib/liblbm_gb300.so``; there is no Python or CPU fallback: if the library
or a CUDA device is missing, the calls raise.

PyTorch supplies device memory (the library's arrays come from PyTorch's
caching allocator through the allocator callbacks of the description) and the
stream (the current torch stream of the device at creation).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbm_gb300.so")
MAX_LEVELS = 4

LBM_OK, LBM_ERR_BAD_DESC, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NEWTON, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
LBM_ERR_ARG = -8
STORAGE = {"f64": 0, "f32": 1, "f16s": 2}
HOLE, BULK, TF_PARENT, HANGING, TF_CHILD = 0, 1, 2, 3, 4

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class lbm_hierarchy_desc(C.Structure):
    _fields_ = [
        ("lattice", C.c_int),
        ("n_levels", C.c_int),
        ("coarse_n", C.c_int64 * 3),
        ("box_lo", (C.c_int64 * 3) * MAX_LEVELS),
        ("box_hi", (C.c_int64 * 3) * MAX_LEVELS),
        ("nu0", C.c_double),
        ("sigma", C.c_double),
        ("dc_variant", C.c_int),
        ("storage", C.c_int),
        ("psi_sign", C.c_int),
        ("use_graphs", C.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", C.c_void_p),
        ("u_shift", C.c_double * 3),
    ]


EXPORTS = [
    "lbm_create_hierarchy", "lbm_create_hierarchy_masked", "lbm_create_error", "lbm_query_level", "lbm_node_class", "lbm_init_fields",
    "lbm_advance", "lbm_get_macros", "lbm_get_pops", "lbm_reduce", "lbm_check_status", "lbm_max_newton_iters",
    "lbm_timing_enable", "lbm_timing_read", "lbm_launch_count", "lbm_device_bytes", "lbm_synchronize",
    "lbm_last_error", "lbm_destroy", "lbm_reduce_static", "lbm_create_batch", "lbm_batch_member",
    "lbm_batch_check_barrier", "lbm_set_probes", "lbm_get_probes", "lbm_save_state", "lbm_load_state",
    "lbm_autotune", "lbm_set_tile_config", "lbm_get_tile_config", "lbm_set_interface_mapping",
    "lbm_reduce_async", "lbm_debug_withhold_copy", "lbm_batch_set_path", "lbm_batch_get_path",
]
TILE_CONFIGS = 5
IFACE_AUTO, IFACE_NODE, IFACE_SEGMENT = 0, 1, 2
BATCH_PERSISTENT, BATCH_PHASES = 0, 1

_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    L = C.CDLL(LIB_PATH)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    L.lbm_create_hierarchy.argtypes = [C.POINTER(lbm_hierarchy_desc), vp, C.POINTER(vp)]
    L.lbm_create_hierarchy_masked.argtypes = [C.POINTER(lbm_hierarchy_desc), C.POINTER(C.c_void_p), vp, C.POINTER(vp)]
    L.lbm_create_error.restype = C.c_char_p
    L.lbm_query_level.argtypes = [vp, C.c_int, i64p, i64p, i64p, dp]
    L.lbm_node_class.argtypes = [vp, C.c_int, vp]
    L.lbm_init_fields.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.lbm_advance.argtypes = [vp, C.c_int64]
    L.lbm_get_macros.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.lbm_get_pops.argtypes = [vp, C.c_int, vp, C.c_int]
    L.lbm_reduce.argtypes = [vp, C.c_int, dp]
    L.lbm_reduce_static.argtypes = [vp, C.c_int, dp]
    L.lbm_reduce_async.argtypes = [vp, C.c_int, vp, C.c_int]
    L.lbm_check_status.argtypes = [vp]
    L.lbm_max_newton_iters.argtypes = [vp]
    L.lbm_timing_enable.argtypes = [vp, C.c_int]
    L.lbm_timing_read.argtypes = [vp, dp, i64p]
    L.lbm_launch_count.argtypes = [vp]
    L.lbm_launch_count.restype = C.c_int64
    L.lbm_device_bytes.argtypes = [vp]
    L.lbm_device_bytes.restype = C.c_int64
    L.lbm_synchronize.argtypes = [vp]
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_create_batch.argtypes = [C.POINTER(lbm_hierarchy_desc), C.c_int, vp, C.POINTER(vp)]
    L.lbm_batch_member.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.lbm_batch_check_barrier.argtypes = [vp, C.c_int, C.c_int64]
    L.lbm_set_probes.argtypes = [vp, C.c_int, dp, C.c_int64]
    L.lbm_get_probes.argtypes = [vp, dp, i64p]
    L.lbm_save_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.lbm_load_state.argtypes = [vp, vp, C.c_size_t]
    L.lbm_autotune.argtypes = [vp, C.c_int, dp]
    L.lbm_set_tile_config.argtypes = [vp, C.c_int, C.c_int]
    L.lbm_set_interface_mapping.argtypes = [vp, C.c_int]
    L.lbm_get_tile_config.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    L.lbm_batch_set_path.argtypes = [vp, C.c_int]
    L.lbm_batch_get_path.argtypes = [vp]
    L.lbm_debug_withhold_copy.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64]
    _lib = L
    return L


def make_desc(desc: dict, use_graphs: bool = True) -> lbm_hierarchy_desc:
    d = lbm_hierarchy_desc()
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
    d.storage = STORAGE[desc.get("storage", "f64")]
    d.psi_sign = int(desc.get("psi_sign", -1))
    d.use_graphs = int(bool(use_graphs))
    us = list(desc.get("u_shift", (0.0, 0.0, 0.0))) + [0.0] * 3
    for a in range(3):
        d.u_shift[a] = float(us[a])
    return d


class _TorchAllocator:
    """Device allocator callbacks backed by PyTorch's caching allocator."""

    def __init__(self, torch, device, stream):
        self._torch, self._dev, self._stream = torch, device, stream

        def _alloc(nbytes, _ctx):
            try:
                return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self._dev, self._stream))
            except Exception:  # out of memory: the library turns NULL into LBM_ERR_OOM
                return None

        def _free(ptr, _ctx):
            if ptr:
                self._torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array, plus on_device flag."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p), 0
    return C.c_void_p(a.data_ptr()), 1


class Hierarchy:
    """Handle of one hierarchy on the current CUDA device (see include/lbm.h)."""

    def __init__(self, desc: dict, use_graphs: bool = True, torch_alloc: bool = True, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the library has no CPU path")
        L = lib()
        self.torch = torch
        self.device = torch.cuda.current_device()
        cur = stream if stream is not None else torch.cuda.current_stream()
        if cur.cuda_stream == 0:
            # the legacy default stream cannot be captured into CUDA graphs: the handle
            # gets a stream of its own, ordered against the caller's stream at every call
            # that takes device tensors
            cur = torch.cuda.Stream()
        self._stream_obj = cur
        self.stream = cur
        d = make_desc(desc, use_graphs)
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(torch, self.device, self._stream_obj.cuda_stream)
            d.alloc, d.free = self._alloc.alloc, self._alloc.free
        self._desc = d
        h = C.c_void_p()
        masks = desc.get("masks")
        if masks is not None and any(m is not None for m in masks[1:]):
            # staircase regions: one byte per parent cell of each level's box, x fastest
            keep = [None if m is None else np.ascontiguousarray(np.asarray(m, dtype=np.uint8)) for m in masks]
            arr = (C.c_void_p * MAX_LEVELS)()
            for l, m in enumerate(keep):
                if l > 0 and m is not None:
                    arr[l] = m.ctypes.data
            rc = L.lbm_create_hierarchy_masked(C.byref(d), arr, C.c_void_p(self._stream_obj.cuda_stream), C.byref(h))
        else:
            rc = L.lbm_create_hierarchy(C.byref(d), C.c_void_p(self._stream_obj.cuda_stream), C.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, L.lbm_create_error().decode())
        self._h = h
        self.q = d.lattice
        self.D = 2 if self.q == 9 else 3
        self.n_levels = d.n_levels
        self.levels = [self.query_level(l) for l in range(self.n_levels)]

    # -------------------------------------------------------------- helpers
    def _enter(self, dev):
        if dev:
            self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self, dev):
        if dev:
            self.torch.cuda.current_stream().wait_stream(self.stream)

    def _check(self, rc):
        if rc != LBM_OK:
            raise LbmError(rc, lib().lbm_last_error(self._h).decode())

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().lbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- C-ABI
    def query_level(self, l):
        n = (C.c_int64 * 3)()
        off = (C.c_int64 * 3)()
        na = C.c_int64()
        tau = C.c_double()
        self._check(lib().lbm_query_level(self._h, l, n, off, C.byref(na), C.byref(tau)))
        return {"n": tuple(n), "off": tuple(off), "n_active": na.value, "tau": tau.value, "N": n[0] * n[1] * n[2]}

    def node_class(self, l):
        out = np.zeros(self.levels[l]["N"], dtype=np.uint8)
        self._check(lib().lbm_node_class(self._h, l, out.ctypes.data_as(C.c_void_p)))
        return out

    def init_fields(self, l, rho, u):
        """rho [N], u [D, N] as float64 numpy arrays (host) or CUDA tensors (device)."""
        N = self.levels[l]["N"]
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.D, N)
        pr, dev = _ptr(rho)
        pu, _ = _ptr(u)
        self._enter(dev)
        self._check(lib().lbm_init_fields(self._h, l, pr, pu, dev))
        self._leave(dev)

    def advance(self, n):
        self._check(lib().lbm_advance(self._h, int(n)))

    def get_macros(self, l, out=None):
        """(rho [N], u [D, N]) as numpy (out=None) or into the given CUDA tensors."""
        N = self.levels[l]["N"]
        if out is None:
            rho = np.zeros(N)
            u = np.zeros((self.D, N))
        else:
            rho, u = out
        pr, dev = _ptr(rho)
        pu, _ = _ptr(u)
        self._enter(dev)
        self._check(lib().lbm_get_macros(self._h, l, pr, pu, dev))
        self._leave(dev)
        return rho, u

    def get_pops(self, l):
        f = np.zeros((self.q, self.levels[l]["N"]))
        self._check(lib().lbm_get_pops(self._h, l, f.ctypes.data_as(C.c_void_p), 0))
        return f

    def reduce(self, l):
        out = (C.c_double * 4)()
        self._check(lib().lbm_reduce(self._h, l, out))
        return np.array(out[:])

    def reduce_async(self, l, out):
        """lbm_reduce_async: enqueue the level's mass and momentum into out (4 float64)
        without synchronising.  out is page-locked host memory (a pinned CPU tensor or a
        numpy view of one) or a CUDA tensor; it holds the sums after synchronize()."""
        if isinstance(out, np.ndarray):
            if out.dtype != np.float64 or out.size < 4 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a contiguous float64 array of at least 4 values")
            ptr, dev = out.ctypes.data_as(C.c_void_p), 0
        else:
            if out.dtype != self.torch.float64 or out.numel() < 4 or not out.is_contiguous():
                raise ValueError("out must be a contiguous float64 tensor of at least 4 values")
            ptr, dev = C.c_void_p(out.data_ptr()), int(out.is_cuda)
        self._enter(dev)
        self._check(lib().lbm_reduce_async(self._h, l, ptr, dev))
        self._leave(dev)

    def reduce_static(self, l):
        """lbm_reduce_static: the same sums with the partials in static device memory."""
        out = (C.c_double * 4)()
        self._check(lib().lbm_reduce_static(self._h, l, out))
        return np.array(out[:])

    def check_status(self):
        self._check(lib().lbm_check_status(self._h))

    def set_probes(self, xyz, capacity):
        """Density probes at points xyz [n, 3] (level-0 units), sampled after every coarse step."""
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        self._n_probes = xyz.shape[0]
        self._check(lib().lbm_set_probes(self._h, xyz.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)),
                                         int(capacity)))

    def get_probes(self):
        n = C.c_int64()
        self._check(lib().lbm_get_probes(self._h, None, C.byref(n)))
        out = np.zeros((n.value, getattr(self, "_n_probes", 0)))
        if out.size:
            self._check(lib().lbm_get_probes(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n)))
        return out

    def save_state(self):
        n = C.c_size_t()
        self._check(lib().lbm_save_state(self._h, None, C.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        self._check(lib().lbm_save_state(self._h, buf.ctypes.data_as(C.c_void_p), C.byref(n)))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(lib().lbm_load_state(self._h, buf.ctypes.data_as(C.c_void_p), buf.size))

    def set_tile_config(self, level, cfg):
        self._check(lib().lbm_set_tile_config(self._h, level, int(cfg)))

    def set_interface_mapping(self, mode):
        """IFACE_AUTO, IFACE_NODE (one interface node per thread) or IFACE_SEGMENT (one
        warp segment per node)."""
        self._check(lib().lbm_set_interface_mapping(self._h, int(mode)))

    def tile_config(self, level):
        c = C.c_int()
        self._check(lib().lbm_get_tile_config(self._h, level, C.byref(c)))
        return c.value

    def autotune(self, reps=20, cache=None):
        """Pick the fastest bulk tile shape per level (lbm_autotune).  With `cache` (a
        JSON file path) results are looked up by (lattice, storage, level boxes) and
        stored after a measurement."""
        import json

        key = json.dumps([self.q, self._desc.storage, [lv["n"] for lv in self.levels]])
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
            if key in table:
                for l, c in enumerate(table[key]["cfg"]):
                    self.set_tile_config(l, c)
                return table[key]
        us = (C.c_double * (self.n_levels * TILE_CONFIGS))()
        self._check(lib().lbm_autotune(self._h, int(reps), us))
        res = {"cfg": [self.tile_config(l) for l in range(self.n_levels)],
               "us": [list(us[l * TILE_CONFIGS:(l + 1) * TILE_CONFIGS]) for l in range(self.n_levels)]}
        if cache:
            table[key] = res
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(table, fh)
            os.replace(tmp, cache)
        return res

    def debug_withhold_copy(self, level, block, k, limit_us):
        """Test hook of the D3Q19 bulk kernel's bounded waits (lbm_debug_withhold_copy):
        block (bx, by, bz) of the level's bulk launches leaves its k-th stage unfilled;
        level < 0 turns it off."""
        bx, by, bz = block
        self._check(lib().lbm_debug_withhold_copy(self._h, int(level), int(bx), int(by), int(bz), int(k),
                                                  int(limit_us)))

    def max_newton_iters(self):
        return lib().lbm_max_newton_iters(self._h)

    def timing_enable(self, on=True):
        self._check(lib().lbm_timing_enable(self._h, int(on)))

    def timing_read(self):
        ms = (C.c_double * MAX_LEVELS)()
        n = (C.c_int64 * MAX_LEVELS)()
        self._check(lib().lbm_timing_read(self._h, ms, n))
        return list(ms[: self.n_levels]), list(n[: self.n_levels])

    def launch_count(self):
        return lib().lbm_launch_count(self._h)

    def device_bytes(self):
        return lib().lbm_device_bytes(self._h)

    def synchronize(self):
        self._check(lib().lbm_synchronize(self._h))


class _Member(Hierarchy):
    """A hierarchy owned by a Batch (no advance of its own)."""

    def __init__(self, batch, handle):  # noqa: D401 - wraps an existing handle
        self.torch = batch.torch
        self.device = batch.device
        self.stream = batch.stream
        self._stream_obj = batch.stream
        self._batch = batch
        self._h = handle
        self._alloc = None
        info = self.query_level(0)
        self.levels = [info]
        n = 1
        while True:
            try:
                self.levels.append(self.query_level(n))
                n += 1
            except LbmError:
                break
        self.n_levels = n
        self.q = 9
        self.D = 2

    def close(self):
        self._h = None  # the batch destroys its members


class Batch:
    """Many independent D2Q9 hierarchies advanced together by one persistent
    cooperative launch per advance() (lbm_create_batch)."""

    def __init__(self, descs, torch_alloc: bool = True, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the library has no CPU path")
        L = lib()
        self.torch = torch
        self.device = torch.cuda.current_device()
        cur = stream if stream is not None else torch.cuda.current_stream()
        if cur.cuda_stream == 0:
            cur = torch.cuda.Stream()
        self.stream = cur
        arr = (lbm_hierarchy_desc * len(descs))()
        self._alloc = _TorchAllocator(torch, self.device, cur.cuda_stream) if torch_alloc else None
        for i, d in enumerate(descs):
            arr[i] = make_desc(d, use_graphs=False)
            if self._alloc:
                arr[i].alloc, arr[i].free = self._alloc.alloc, self._alloc.free
        self._descs = arr
        h = C.c_void_p()
        rc = L.lbm_create_batch(arr, len(descs), C.c_void_p(cur.cuda_stream), C.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, L.lbm_create_error().decode())
        self._h = h
        self.members = []
        for i in range(len(descs)):
            m = C.c_void_p()
            self._check(L.lbm_batch_member(h, i, C.byref(m)))
            self.members.append(_Member(self, m))

    def _check(self, rc):
        if rc != LBM_OK:
            raise LbmError(rc, lib().lbm_last_error(self._h).decode())

    def advance(self, n):
        self._check(lib().lbm_advance(self._h, int(n)))

    def check_status(self):
        self._check(lib().lbm_check_status(self._h))

    def set_path(self, path):
        """BATCH_PERSISTENT (one cooperative launch per coarse step) or BATCH_PHASES (one
        launch per phase)."""
        self._check(lib().lbm_batch_set_path(self._h, int(path)))

    def path(self):
        return lib().lbm_batch_get_path(self._h)

    def autotune(self, reps=5):
        """Time both launch structures over reps coarse steps of the live state and keep
        the faster (the state advances: initialise the members afterwards)."""
        us = (C.c_double * 2)()
        self._check(lib().lbm_autotune(self._h, int(reps), us))
        return {"path": self.path(), "us": [us[0], us[1]]}

    def check_barrier(self, skip_block, limit_us):
        return lib().lbm_batch_check_barrier(self._h, int(skip_block), int(limit_us))

    def launch_count(self):
        return lib().lbm_launch_count(self._h)

    def device_bytes(self):
        return lib().lbm_device_bytes(self._h) + sum(m.device_bytes() for m in self.members)

    def synchronize(self):
        self._check(lib().lbm_synchronize(self._h))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            for m in self.members:
                m._h = None
            lib().lbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
