#!/usr/bin/env python
"""Throughput of the multi-level DC2 / H-RR lattice Boltzmann hot path on GB300.

Headline workload (the largest single-GPU configuration): the D3Q19 three-level
slab hierarchy, coarse 512x512x256, a level-1 slab spanning x and y (z in
[96,160)) and a level-2 box [128,384)^2 x [112,144), 0.305 G active nodes, an
acoustic pulse (1e-4) and a vortex in a Mach-0.15 mean flow, FP16 storage of
f_i - w_i with FP32 arithmetic.  One step = one coarse step = 1 step of level 0,
2 of level 1 and 4 of level 2 (0.83 G node updates, 17.2 G fine-equivalent).
FP64, FP32 and FP16 of f_i - f_i^eq(1, U) are reported beside it ("variants"),
and the other configurations each with their own roofline ("extras").  Inputs
live in HBM when timing starts; the L2 is flushed (256 MB write) before every
timed step, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload W] [--storage S]

For N > 1 (torchrun) every rank advances an independent replica of the same
hierarchy (the single hierarchy does not shard; replicas only); the value is
the sum of the ranks' node updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (fine-equiv) & % HBM roofline, FP32/FP16-shift vs FP64 on same GB300"
UNIT = "MLUPS (fine-equivalent)"
BYTES_PER_POP = {"f64": 8, "f32": 4, "f16s": 2, "f16s_mean": 2}


def _with_storage(d, storage):
    """A description in one of the reported storage forms: f64, f32, f16s (half of
    f_i - w_i) or f16s_mean (half of f_i - f_i^eq(1, U), U the workload's mean flow)."""
    d = dict(d)
    if storage == "f16s_mean":
        d["storage"] = "f16s"
        d["u_shift"] = tuple(d["init"]["U"])
    else:
        d["storage"] = storage
        d.pop("u_shift", None)
    return d


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the default process group (x itself when there
    is none): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, seconds):
    """Units per second of the whole job: every rank processes units_per_rank
    (independent replicas), the job lasts as long as its slowest rank."""
    return world_size * units_per_rank / seconds


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOAD_TEXT = {
    "pulse2d_3lvl": "pulse2d_3lvl: D2Q9, 3 levels, coarse 512^2 periodic, patches 256^2 and 128^2 coarse cells, "
                    "Mach 0.2, A=1e-3",
    "vortex2d_2lvl": "vortex2d_2lvl: D2Q9, 2 levels, coarse 128^2 periodic, patch 64^2 coarse cells, vortex at Mach 0.1",
    "vortex3d_3lvl": "vortex3d_3lvl: D3Q19, 3 levels, coarse 256^3 periodic, cubes 128^3 and 64^3 coarse cells, "
                     "vortex tube + 1% noise at Mach 0.1",
    "slab3d_3lvl": "slab3d_3lvl: D3Q19, 3 levels, coarse 512x512x256, slab z in [96,160) and box "
                   "[128,384)^2 x [112,144), pulse 1e-4 + vortex at Mach 0.15",
    "vortex3d_3lvl_128": "vortex3d_3lvl_128: D3Q19, 3 levels, coarse 128^3 periodic, cubes 64^3 and 32^3 coarse "
                         "cells (half-size replica of vortex3d_3lvl, for profiling)",
    "slab3d_3lvl_256": "slab3d_3lvl_256: D3Q19, 3 levels, coarse 256x256x128, slab z in [48,80) and box "
                       "[64,192)^2 x [56,72) (half-size replica of slab3d_3lvl per axis, for profiling)",
    "batch2d": "batch2d: 96 independent D2Q9 2-level hierarchies, coarse sides drawn from {96..1024}, centred "
               "patches of half the side, seeded vortices or pulses, one persistent cooperative launch per step",
}
DEFAULT_STORAGE = {"pulse2d_3lvl": "f32", "vortex2d_2lvl": "f64", "vortex3d_3lvl": "f32", "slab3d_3lvl": "f16s",
                   "slab3d_3lvl_256": "f16s", "vortex3d_3lvl_128": "f32", "batch2d": "f32"}
DEFAULT_WORKLOAD = "slab3d_3lvl"


def _workloads():
    from paper_2004_14887_gb300 import workloads as W

    return {"pulse2d_3lvl": W.pulse2d, "vortex2d_2lvl": W.vortex2d, "vortex3d_3lvl": W.vortex3d,
            "slab3d_3lvl": W.slab3d,
            "slab3d_3lvl_256": lambda **kw: W.slab3d(nxy=256, nz=128, slab=(48, 80), box=((64, 64, 56), (192, 192, 72)),
                                                     **kw),
            "vortex3d_3lvl_128": lambda **kw: W.vortex3d(n=128, boxes=((32, 96), (48, 80)), **kw),
            "batch2d": W.batch2d}


def kernel_source_key(csrc):
    """Hash of the library sources (kernels, device headers and the host code that
    chooses launch shapes) with comments and blank lines removed: a traffic figure
    measured by ncu stays valid while the code is unchanged."""
    import hashlib

    h = hashlib.sha1()
    for name in sorted(f for f in os.listdir(csrc) if f.endswith((".cuh", ".cu"))):
        txt = open(os.path.join(csrc, name)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update("\n".join(ln.rstrip() for ln in txt.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:12]


def _traffic_from_profiles(workload, storage):
    """DRAM bytes per launch recorded by an ncu capture in profiles/ for this kernel,
    workload and kernel-source revision, or None."""
    path = os.path.join(ROOT, "profiles", f"k_bulk_{workload}_{storage}.md")
    if not os.path.exists(path):
        return None
    try:
        from paper_2004_14887_gb300 import build as B

        import hashlib

        sha = kernel_source_key(B.CSRC)
        txt = open(path).read()
        m = re.search(r"traffic_per_full_launch_bytes:\s*([0-9.eE+]+)\s+source_sha:\s*(\w+)", txt)
        if m and m.group(2) == sha:
            return float(m.group(1))
    except Exception:
        return None
    return None


_FIELDS = {}


def _fields(d, l):
    """Initial (rho, u) of level l of a workload, computed once per (workload, level)
    and shared by every hierarchy of the run built from it (storage forms differ only
    in how the library stores the same state)."""
    from paper_2004_14887_gb300 import workloads as W

    key = (d.get("name"), json.dumps(d["boxes"]), json.dumps(d["init"], sort_keys=True), l)
    if key not in _FIELDS:
        _FIELDS[key] = W.init_fields(d, l)
    return _FIELDS[key]


def _flush_buffer():
    import torch

    return torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def measure_hierarchy(workload, storage, K, Wm, flush, *, sampler_dev=None, autotune=True, ws=1, timing_steps=None,
                      label=None):
    """Device-timed coarse steps of one hierarchy (CUDA events on the library's stream
    around every step, the L2 flushed before each, outside the events) and the
    average duration of the dominant kernel, the finest level's bulk collide-and-stream
    launch (the library's per-launch CUDA events, lbm_timing_*)."""
    import torch

    from paper_2004_14887_gb300 import lbm
    from paper_2004_14887_gb300 import workloads as W

    d = _with_storage(_workloads()[workload](), storage)
    tc = time.perf_counter()
    h = lbm.Hierarchy(d)
    setup_s = time.perf_counter() - tc
    tuned = None
    if autotune:
        tuned = h.autotune(reps=10)["cfg"]
    for l in range(h.n_levels):
        r, u = _fields(d, l)
        h.init_fields(l, r, u)
    print(f"[bench] {label or workload} {storage}: set-up {setup_s:.2f} s, {h.device_bytes() / 1e9:.2f} GB on the "
          f"device, tile configurations {tuned}", file=sys.stderr, flush=True)
    h.advance(Wm)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    n0 = h.launch_count()
    _barrier(ws)
    torch.cuda.synchronize()
    clocks = None

    def loop():
        for k in range(K):
            flush.zero_()
            starts[k].record()
            h.advance(1)
            ends[k].record()
        torch.cuda.synchronize()

    if sampler_dev is not None:
        with ClockSampler(sampler_dev) as cs:
            loop()
        clocks = cs.summary()
    else:
        loop()
    _barrier(ws)
    h.check_status()
    dev_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    launches = h.launch_count() - n0
    t = max_over_ranks(dev_ms, device="cuda") / 1e3
    upd = W.updates_per_coarse_step(d)
    feq = W.fine_equivalent_per_coarse_step(d)
    L = h.n_levels
    # dominant kernel: the bulk collide-and-stream launch of the finest level
    h.timing_enable(True)
    for _ in range(timing_steps or min(K, 200)):
        flush.zero_()
        h.advance(1)
    ms, cnt = h.timing_read()
    h.timing_enable(False)
    bulk_ms = [m / max(c, 1) for m, c in zip(ms, cnt)]
    nact = [h.levels[l]["n_active"] for l in range(L)]
    bpp = BYTES_PER_POP[storage]
    bytes_finest = nact[L - 1] * 2 * h.q * bpp
    peak, peak_src = _peaks()
    achieved = bytes_finest / (bulk_ms[L - 1] * 1e-3) / 1e9
    kname = "k_bulk3d" if h.q == 19 else "k_bulk2d"
    out = {
        "value": ws * feq * K / t / 1e6, "actual_mlups": ws * upd * K / t / 1e6, "ms_per_step": 1e3 * t / K,
        "steps": K, "warmup": Wm, "storage": storage, "gpu_launches": launches, "clocks": clocks,
        "node_updates_per_step": upd, "fine_equivalent_updates_per_step": feq, "active_nodes_per_level": nact,
        "bulk_ms_per_launch_by_level": bulk_ms, "tile_config_per_level": tuned,
        "device_bytes": h.device_bytes(), "setup_s": setup_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic_from_profiles(workload, storage),
                     "kernel": f"{kname}, bulk collide-and-stream of the finest level (level {L - 1}, "
                               f"{nact[L - 1]} active nodes, {2 ** (L - 1)} launches per step)",
                     "algorithmic_bytes_per_launch": bytes_finest, "avg_launch_ms": bulk_ms[L - 1],
                     "peak_source": f"{peak_src} hbm_gbs (of {peak_src})"},
        "step_roofline_frac": upd * 2 * h.q * bpp / (t / K) / 1e9 / peak,
    }
    h.close()
    del h
    torch.cuda.synchronize()
    return out


def measure_batch(storage, K, Wm, flush, *, sampler_dev=None, ws=1):
    """The batched workload: every step advances all hierarchies of the batch by one
    coarse step in one cooperative persistent launch."""
    import torch

    from paper_2004_14887_gb300 import lbm
    from paper_2004_14887_gb300 import workloads as W

    descs = [_with_storage(d, storage) for d in W.batch2d()]
    tc = time.perf_counter()
    b = lbm.Batch(descs)
    for d, m in zip(descs, b.members):
        for l in range(m.n_levels):
            r, u = _fields(d, l)
            m.init_fields(l, r, u)
    # launch structure chosen by the autotuner (it advances the state: initialise again)
    tuned = b.autotune(reps=3)
    for d, m in zip(descs, b.members):
        for l in range(m.n_levels):
            r, u = _fields(d, l)
            m.init_fields(l, r, u)
    print(f"[bench] batch2d {storage}: {len(descs)} hierarchies, set-up {time.perf_counter() - tc:.2f} s, "
          f"{b.device_bytes() / 1e9:.2f} GB on the device", file=sys.stderr, flush=True)
    upd = sum(W.updates_per_coarse_step(d) for d in descs)
    feq = sum(W.fine_equivalent_per_coarse_step(d) for d in descs)
    b.advance(Wm)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    n0 = b.launch_count()
    _barrier(ws)
    torch.cuda.synchronize()
    clocks = None

    def loop():
        for k in range(K):
            flush.zero_()
            starts[k].record()
            b.advance(1)
            ends[k].record()
        torch.cuda.synchronize()

    if sampler_dev is not None:
        with ClockSampler(sampler_dev) as cs:
            loop()
        clocks = cs.summary()
    else:
        loop()
    _barrier(ws)
    b.check_status()
    ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    t = max_over_ranks(ms, device="cuda") / 1e3
    peak, peak_src = _peaks()
    bytes_step = upd * 2 * 9 * BYTES_PER_POP[storage]
    out = {
        "value": ws * feq * K / t / 1e6, "actual_mlups": ws * upd * K / t / 1e6, "ms_per_step": 1e3 * t / K,
        "steps": K, "warmup": Wm, "storage": storage, "hierarchies": len(descs), "gpu_launches": b.launch_count() - n0,
        "launch_structure": {"chosen": "phases" if tuned["path"] == lbm.BATCH_PHASES else "persistent",
                             "us_per_step_persistent": tuned["us"][0], "us_per_step_phases": tuned["us"][1]},
        "clocks": clocks, "node_updates_per_step": upd, "fine_equivalent_updates_per_step": feq,
        "roofline": {"bound": "hbm", "achieved": bytes_step / (t / K) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bytes_step / (t / K) / 1e9 / peak, "traffic": None,
                     "kernel": "whole coarse step (k_batch, or k_batch_bulk / k_batch_rh / k_batch_gi per phase)",
                     "algorithmic_bytes_per_launch": bytes_step, "avg_launch_ms": 1e3 * t / K,
                     "peak_source": f"{peak_src} hbm_gbs (of {peak_src})"},
    }
    b.close()
    torch.cuda.synchronize()
    return out


def measure_e2e(workload, storage, K, ws=1):
    """End to end through the public API with host buffers: the initial fields from
    pinned host memory (H2D), then every step advances and copies the finest level's
    FP64 mass and momentum into its row of a pinned host array (D2H, lbm_reduce_async,
    stream-ordered), and at the end the macros of every level (D2H, synchronising);
    the handle is set up as a user would: created, initialised, autotuned."""
    import torch

    from paper_2004_14887_gb300 import lbm
    from paper_2004_14887_gb300 import workloads as W

    de = _with_storage(_workloads()[workload](), storage)
    he = lbm.Hierarchy(de)
    fields = []
    for l in range(he.n_levels):
        r, u = _fields(de, l)
        rp = torch.from_numpy(r).pin_memory().numpy()
        up = torch.from_numpy(u).pin_memory().numpy()
        fields.append((rp, up))
        he.init_fields(l, rp, up)
    he.autotune(reps=10)
    outs = [(torch.empty(he.levels[l]["N"], dtype=torch.float64).pin_memory().numpy(),
             torch.empty((he.D, he.levels[l]["N"]), dtype=torch.float64).pin_memory().numpy())
            for l in range(he.n_levels)]
    sums = torch.zeros((K, 4), dtype=torch.float64).pin_memory()
    # warm-up on the workload's own state (graph capture); the timed region starts
    # again from the initial fields
    he.advance(3)
    he.check_status()
    torch.cuda.synchronize()
    _barrier(ws)
    te = time.perf_counter()
    for l in range(he.n_levels):
        he.init_fields(l, *fields[l])
    for k in range(K):
        he.advance(1)
        he.reduce_async(he.n_levels - 1, sums[k])
    for l in range(he.n_levels):
        he.get_macros(l, out=outs[l])
    torch.cuda.synchronize()
    _barrier(ws)
    tw = max_over_ranks(time.perf_counter() - te, device="cuda")
    he.check_status()
    if not bool(torch.isfinite(sums).all()):
        raise RuntimeError("end-to-end run: non-finite mass or momentum")
    h2d = sum(a.nbytes + b.nbytes for a, b in fields)
    d2h = sum(a.nbytes + b.nbytes for a, b in outs) + sums.numel() * 8
    feq = W.fine_equivalent_per_coarse_step(de)
    he.close()
    del he, outs, fields
    torch.cuda.synchronize()
    return {"value": ws * feq * K / tw / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K,
            "per_step": "advance one coarse step + FP64 mass/momentum of the finest level into a pinned host row "
                        "(stream-ordered, no per-step synchronisation); initial fields H2D and final macros D2H "
                        "amortised over the steps; no L2 flush between steps"}


def bulk_at_scale(storage, flush):
    """The 2-D bulk kernel on one large level (4096^2, 1.2 GB per launch in FP32),
    where the launch is long enough for HBM to be the limit."""
    import torch

    from paper_2004_14887_gb300 import lbm
    from paper_2004_14887_gb300 import workloads as W

    n = 4096
    ds = {"lattice": 9, "coarse_n": (n, n), "boxes": [], "nu0": 1e-5, "storage": storage,
          "init": {"kind": "vortex", "xc": n / 2, "yc": n / 2, "Rc": n / 16, "swirl": 0.05, "U": (0.05, 0.02, 0.0)}}
    hs = lbm.Hierarchy(ds)
    r, u = W.init_fields(ds, 0)
    hs.init_fields(0, r, u)
    hs.autotune(reps=5)
    hs.advance(3)
    torch.cuda.synchronize()
    ks = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hs.advance(ks)
    e1.record()
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1) / ks
    bytes_s = n * n * 2 * 9 * BYTES_PER_POP[storage]
    hs.close()
    return {"workload": f"single periodic D2Q9 level {n}^2, {storage}, vortex", "ms_per_launch": ms_s,
            "achieved_gbs": bytes_s / (ms_s * 1e-3) / 1e9, "frac": bytes_s / (ms_s * 1e-3) / 1e9 / _peaks()[0],
            "mlups": n * n / (ms_s * 1e-3) / 1e6}


# the other configurations, each reported beside the headline with its own roofline:
# (workload, storage, timed steps)
EXTRAS = [("pulse2d_3lvl", "f32", 200), ("pulse2d_3lvl", "f16s_mean", 200), ("vortex3d_3lvl", "f32", 20),
          ("batch2d", "f32", 20)]


def run_gb300(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    # one non-default stream for the library, the L2 flushes and the timing events
    torch.cuda.set_stream(torch.cuda.Stream())
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    flush = _flush_buffer()
    K, Wm = args.steps, args.warmup
    main_storage = args.storage or DEFAULT_STORAGE[args.workload]
    if args.workload == "batch2d":
        main = measure_batch(main_storage, K, Wm, flush, sampler_dev=local, ws=ws)
    else:
        main = measure_hierarchy(args.workload, main_storage, K, Wm, flush, sampler_dev=local,
                                 autotune=not args.no_autotune, ws=ws)

    # the other storage forms of the same workload (FP64 with few steps: it is the
    # slow reference of the speed-up)
    variants = {}
    if not args.no_variants and args.workload != "batch2d":
        for st in [x for x in ("f64", "f32", "f16s", "f16s_mean") if x != main_storage]:
            Kv = min(K, args.variant_steps) if st == "f64" else K
            v = measure_hierarchy(args.workload, st, Kv, min(Wm, 3), flush, autotune=not args.no_autotune, ws=ws,
                                  timing_steps=min(Kv, 20))
            variants[st] = {k: v[k] for k in ("value", "actual_mlups", "ms_per_step", "steps")}
            variants[st]["finest_bulk_gbs"] = v["roofline"]["achieved"]
            variants[st]["finest_bulk_frac"] = v["roofline"]["frac"]
        vals = {k: v["value"] for k, v in variants.items()}
        vals[main_storage] = main["value"]
        for st in ("f32", "f16s", "f16s_mean"):
            if st in vals and "f64" in vals:
                variants[f"{st}_speedup_vs_f64"] = vals[st] / vals["f64"]

    extras = {}
    if not args.no_extras and ws == 1:
        for wl, st, ke in EXTRAS:
            if wl == args.workload and st == main_storage:
                continue
            key = f"{wl}_{st}"
            if wl == "batch2d":
                extras[key] = measure_batch(st, ke, 5, flush)
            else:
                extras[key] = measure_hierarchy(wl, st, ke, 5, flush, timing_steps=min(ke, 50))
            extras[key]["workload"] = WORKLOAD_TEXT[wl] + f", {st} storage"
        if not args.no_scale_check:
            extras["bulk_at_scale_f32"] = bulk_at_scale("f32", flush)
            extras["bulk_at_scale_f16s"] = bulk_at_scale("f16s", flush)

    e2e = None
    if not args.no_e2e and args.workload != "batch2d":
        e2e = measure_e2e(args.workload, main_storage, K, ws=ws)

    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
        "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": main_storage, "data": "synthetic (seeded analytic fields, no dataset)",
        "config": {"workload": WORKLOAD_TEXT[args.workload] + f", {main_storage} storage",
                   "node_updates_per_step": main["node_updates_per_step"],
                   "fine_equivalent_updates_per_step": main["fine_equivalent_updates_per_step"],
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "actual_mlups": main["actual_mlups"],
        "roofline": main["roofline"],
        "gpu_launches": main["gpu_launches"],
        "clocks": main["clocks"],
        "e2e": e2e,
    }
    for k in ("active_nodes_per_level", "bulk_ms_per_launch_by_level", "step_roofline_frac", "tile_config_per_level",
              "device_bytes", "setup_s", "hierarchies"):
        if k in main:
            line[k] = main[k]
    line["variants"] = variants
    line["extras"] = extras
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_steps)
        line["cpu_baseline_all_cores"] = cpu_baseline(args.workload, args.cpu_steps, threaded=True)
        forms = [main_storage] + [x for x in variants if "speedup" not in x]
        line["accuracy"] = accuracy(args.workload, forms)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# Bounded samples for the oracle (CPU baseline, reference arm, accuracy): a replica of
# each workload with the same proportions and physics, the coarse steps that keep the
# single-threaded oracle within ~10-30 s, and the steps of the accuracy comparison.
REPLICA = {
    "pulse2d_3lvl": ("128^2 three-level replica (1/4 of each axis)", 150, 40),
    "vortex2d_2lvl": ("full-size 128^2 two-level hierarchy (no replica needed)", 150, 40),
    "vortex3d_3lvl": ("32^3 three-level replica (1/8 of each axis)", 15, 6),
    "vortex3d_3lvl_128": ("32^3 three-level replica (1/8 of vortex3d_3lvl per axis)", 15, 6),
    "slab3d_3lvl": ("64x64x32 three-level replica (1/8 of each axis)", 4, 2),
    "slab3d_3lvl_256": ("64x64x32 three-level replica (1/8 of slab3d_3lvl per axis)", 4, 2),
    "batch2d": ("one 128^2 two-level member", 150, 40),
}


def _replica_desc(workload="slab3d_3lvl", storage="f64"):
    """The replica of a workload on which the oracle is timed and compared."""
    from paper_2004_14887_gb300 import workloads as W

    if workload in ("vortex3d_3lvl", "vortex3d_3lvl_128"):
        return W.vortex3d(n=32, boxes=((8, 24), (12, 20)), storage=storage)
    if workload in ("slab3d_3lvl", "slab3d_3lvl_256"):
        return W.slab3d(nxy=64, nz=32, slab=(12, 20), box=((16, 16, 14), (48, 48, 18)), storage=storage)
    if workload == "vortex2d_2lvl":
        return W.vortex2d(storage=storage)
    if workload == "batch2d":
        return W.batch2d(n=1, sides=(128,), storage=storage)[0]
    return W.pulse2d(n=128, boxes=((32, 96), (48, 80)), steps=20, storage=storage)


def _oracle_run(d, steps, warm=1, threaded=False):
    from oracle import oracle as O

    o = O.Hierarchy(d, threaded=threaded)
    for l in range(o.n_levels):
        r, u = _fields(d, l)
        o.init(l, r, u)
    o.advance(warm)
    t0 = time.perf_counter()
    o.advance(steps)
    return o, time.perf_counter() - t0


def cpu_baseline(workload, steps=None, threaded=False):
    """The FP64 oracle timed on the workload's replica: its plain build
    (single-threaded), or with threaded=True its OpenMP build on every host core
    (the same per-node arithmetic, the node loops shared out over threads)."""
    from paper_2004_14887_gb300 import workloads as W

    text, default_steps, _ = REPLICA[workload]
    steps = steps or default_steps
    cores = 1
    if threaded:
        from oracle import oracle as O

        cores = O.threads(os.cpu_count() or 1)
    d = _replica_desc(workload)
    _, dt = _oracle_run(d, steps, threaded=threaded)
    feq = W.fine_equivalent_per_coarse_step(d)
    how = f"OpenMP FP64 oracle on {cores} host threads" if threaded else "single-threaded FP64 oracle"
    return {"value": feq * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} coarse steps of the {text} of the workload "
                      f"({W.updates_per_coarse_step(d)} node updates per step), {how}",
            "actual_mlups": W.updates_per_coarse_step(d) * steps / dt / 1e6}


# pressure scale of the Pa-equivalent error: p' = (rho'/rho0) rho0 c0^2 with
# rho0 c0^2 = 1.206e5 Pa (air at rest); levels in dB re 2e-5 Pa (the usual acoustic
# reference, which the paper does not state)
P_REF_PA = 1.206e5
P_DB_REF_PA = 2e-5


def _db(p_pa):
    import math

    return 20.0 * math.log10(p_pa / P_DB_REF_PA) if p_pa > 0 else float("-inf")


def _storage_error(d, st, steps, o):
    """Advance description d in storage st on the GPU and compare every level with the
    oracle o: (rel Linf rho, rel Linf u, max|drho|, volume-weighted sum drho^2, total
    weight, max|rho - 1| of the oracle)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2004_14887_gb300 import lbm

    d = _with_storage(d, st)
    g = lbm.Hierarchy(d)
    for l in range(g.n_levels):
        r, u = _fields(d, l)
        g.init_fields(l, r, u)
    g.advance(steps)
    g.check_status()
    er = eu = ed = 0.0
    sq, wsum, amp = 0.0, 0.0, 0.0
    L = g.n_levels - 1
    for l in range(g.n_levels):
        m = o.node_class(l) != O.HOLE
        rg, ug = g.get_macros(l)
        ro, uo = o.macros(l)
        amp = max(amp, float(np.max(np.abs(ro[m] - 1.0))))
        dr = rg[m] - ro[m]
        er = max(er, float(np.max(np.abs(dr)) / np.max(np.abs(ro[m]))))
        eu = max(eu, float(np.max(np.abs(ug[:, m] - uo[:, m])) / max(np.max(np.abs(uo[:, m])), 1e-300)))
        ed = max(ed, float(np.max(np.abs(dr))))
        wv = float(1 << (g.D * (L - l)))  # cell volume in finest-level cells
        sq += wv * float(np.sum(dr * dr))
        wsum += wv * dr.size
    g.close()
    return er, eu, ed, sq, wsum, amp


def _all_fine(d):
    """Uniform periodic grid at the finest spacing of d over the same domain (level 0
    of the result has tau_L: nu = 2^L nu_0), with the same analytic fields; one of its
    steps is one finest-level step of d."""
    L = len(d["boxes"])
    f = 1 << L
    D = 2 if d["lattice"] == 9 else 3
    u = dict(d)
    u["boxes"] = []
    u["coarse_n"] = tuple(int(c) * f for c in d["coarse_n"][:D])
    u["nu0"] = d["nu0"] * f
    ini = dict(d["init"])
    for k in ("xc", "yc", "zc", "Rc"):
        if k in ini:
            ini[k] = ini[k] * f
    u["init"] = ini
    u["name"] = (d.get("name") or "replica") + "_all_fine"
    return u, f


def accuracy(workload, storages):
    """The workload's replica advanced on the GPU in each storage and by the FP64
    oracle for the same steps: per storage, the relative L-infinity errors of rho and
    u (worst level), the density error relative to the signal amplitude max|rho - 1|,
    and the volume-weighted RMS density error as a pressure in Pa-equivalent and in dB.
    The same comparison on an all-fine uniform grid at the finest spacing over the same
    physical time (2^L steps per coarse step) gives the storage's own precision floor
    without any interface; floor_ratio = RMS error of the refined run / that floor."""
    text, _, steps = REPLICA[workload]
    d64 = _replica_desc(workload)
    o, _ = _oracle_run(d64, steps, warm=0, threaded=True)
    du, f = _all_fine(d64)
    ou, _ = _oracle_run(du, steps * f, warm=0, threaded=True)
    out = {}
    for st in storages:
        er, eu, ed, sq, wsum, amp = _storage_error(d64, st, steps, o)
        _, _, _, squ, wsu, _ = _storage_error(du, st, steps * f, ou)
        rms = (sq / max(wsum, 1)) ** 0.5
        floor = (squ / max(wsu, 1)) ** 0.5
        out[st] = {"rho_rel_linf": er, "u_rel_linf": eu, "drho_rel_amplitude": ed / max(amp, 1e-300),
                   "dp_rms_pa": rms * P_REF_PA, "dp_rms_db": _db(rms * P_REF_PA), "dp_max_pa": ed * P_REF_PA,
                   "amplitude_pa": amp * P_REF_PA, "amplitude_db": _db(amp * P_REF_PA),
                   "floor_dp_rms_pa": floor * P_REF_PA,
                   "floor_ratio": rms / floor if floor > 0 else (0.0 if rms == 0 else float("inf"))}
    return {"vs": "FP64 oracle", "sample": f"{steps} coarse steps of the {text}",
            "floor": f"the same comparison on an all-fine uniform grid at the finest spacing ({f}x each axis of "
                     f"level 0), {steps * f} steps (the same physical time), against the all-fine oracle",
            "rms": "volume-weighted over the active nodes of every level (weight: cell volume)",
            "db_ref_pa": P_DB_REF_PA, "by_storage": out}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands (its plain,
    single-threaded build) timed on a bounded sample of the same workload (its
    replica), on rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2004_14887_gb300 import workloads as W

    text, _, _ = REPLICA[args.workload]
    K = args.steps
    d = _replica_desc(args.workload)
    _, dt = _oracle_run(d, K, warm=min(args.warmup, 2))
    feq = W.fine_equivalent_per_coarse_step(d)
    v = feq * K / dt / 1e6
    sample = f"{K} coarse steps of the {text} of the workload, single-threaded FP64 oracle"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded analytic fields, no dataset)",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--storage", default=None, choices=["f64", "f32", "f16s", "f16s_mean"])
    ap.add_argument("--variant-steps", type=int, default=5, help="timed steps of the FP64 variant")
    ap.add_argument("--cpu-steps", type=int, default=None, help="oracle steps of the CPU baseline (default per workload)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-scale-check", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
