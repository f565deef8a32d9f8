"""Benchmark of the hybrid PIC ion loop: ion pushes per second including the
periodic sort, the deposit and the full subcycled field advance, on the 2D
Harris-sheet workload (1024x512 cells, dx = 0.25 d_i, 100 ions per cell,
52,428,800 FP32 ions), plus its HBM roofline fraction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole hot path (sort every 8 steps, gather +
Boris push + half-step deposit + move, moment post, 10 field subcycles of
two Ohm/Faraday stages, final Ohm).  Under torchrun each rank runs an
independent replica (the path is not sharded); rank 0 prints one JSON line.
The reference arm times the FP64 CPU oracle on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ion pushes/s incl. deposit+field on 1 GB300"
UNIT = "pushes/s"
PAPER_PUSHES_PER_CORE = 1.0e7  # Sec. 1: ~10 million pushes/s/processor on CPUs


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="harris2d",
                    choices=["harris2d", "harris2d_small", "alfven2d", "beam3d_small", "beam3d",
                             "beam3d_2ppc", "harris3d", "harris3d_quarter", "ebeam2d",
                             "slab2d_open"])
    ap.add_argument("--shape", default="qs", choices=["qs", "cic", "ngp"])
    ap.add_argument("--sort-every", type=int, default=None,
                    help="override the workload's sort interval")
    ap.add_argument("--smooth", type=int, default=0,
                    help="binomial passes on the moments and on the gathered E, B "
                         "(self-consistent smoothing, Sec. 2.2)")
    ap.add_argument("--pe-eq", action="store_true",
                    help="electron energy equation (Sec. 2.1) with gamma_e = 5/3 and "
                         "kappa = 0.01 instead of the equation of state")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--per-step", type=int, default=0,
                    help="instead of the benchmark: profile this many single steps after "
                         "the warm-up and print the push time against the steps since "
                         "the last sort")
    return ap.parse_args()


def make_workload(name, shape, seed_offset=0):
    from paper_2305_05600_gb300 import inputs as I
    # The windowed counting sort costs about 1.5 ms per call at 1024x512; the
    # push is fastest mid-interval, where the ions have reached the cells
    # they were sorted by (predicted 0.6875 intervals ahead).  Sorting every
    # 8 steps minimises the sum (measured on GB300 for 4, 6, 8).
    if name == "harris2d":
        return I.harris(shape=shape, seed=1000 + seed_offset, sort_every=8)
    if name == "harris2d_small":  # ncu-sized case: 13.1M ions, > L2
        return I.harris(nx=512, nz=256, shape=shape, seed=1000 + seed_offset, sort_every=8)
    if name == "alfven2d":
        return I.alfven2d(shape=shape, seed=seed_offset)
    if name == "beam3d_small":
        return I.beam3d(nx=64, ny=64, nz=64, shape=shape, seed=2000 + seed_offset)
    if name == "beam3d":  # 256x128x128 cells, 64 ppc, 268M ions
        return I.beam3d(shape=shape, seed=2000 + seed_offset)
    if name == "beam3d_2ppc":  # the beam grid with 1 core + 1 beam ion per cell (field kernels)
        return I.beam3d(n_core=1, n_beam=1, shape=shape, seed=2000 + seed_offset)
    if name == "harris3d":  # 512x256x256 cells, 32 ppc, 1.07e9 ions, generated on the GPU
        return I.harris_device(shape=shape, seed=3000 + seed_offset)
    if name == "harris3d_quarter":  # 256x128x128 cells, 32 ppc, 134M ions, generated on the GPU
        return I.harris_device(nx=256, ny=128, nz=128, shape=shape, seed=3000 + seed_offset)
    if name == "ebeam2d":  # relativistic electron beam, resistive background, 640x320, 13.1M
        return I.ebeam2d(shape=shape, seed=8000 + seed_offset)
    if name == "slab2d_open":  # plasma flowing through faces open in x, injection, 52.4M ions
        return I.drifting_slab(nx=1024, nz=512, ppc=100, dx=0.25, U=0.4, Ti=0.04, Te=0.02,
                               dt=0.02, nsub=10, shape=shape, open_faces=1, sort_every=4,
                               seed=9000 + seed_offset)
    raise ValueError(name)


def apply_overrides(wl, args):
    if args.sort_every is not None:
        wl.params["sort_every"] = args.sort_every
    if args.smooth:
        wl.params["smooth_passes"] = args.smooth
        wl.params["field_smooth_passes"] = args.smooth
    if args.pe_eq:
        wl.params.update(pe_eq=1, kappa=0.01, gamma_e=5.0 / 3.0)
    return wl


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, enabled: bool):
        self.proc = None
        self.device = device
        if enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(device), f"--query-gpu={self.QUERY}",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# roofline bookkeeping
# ----------------------------------------------------------------------------

def push_bytes_per_launch(wl) -> float:
    """Algorithmic bytes of one push launch: every ion read once (cell, 2 or
    3 offsets, v, w) and written once (all but w), plus, per interior cell,
    E and B read once (24 B) and n, J written once (16 B)."""
    p = wl.params
    dim2 = p["ny"] == 1
    per_ion = (4 + 4 * (2 if dim2 else 3) + 12 + 4) + (4 + 4 * (2 if dim2 else 3) + 12)
    ncell = p["nx"] * p["ny"] * p["nz"]
    return float(wl.n_particles * per_ion + ncell * (24 + 16))


def step_bytes(wl) -> dict:
    """Algorithmic bytes of one whole step: the push's (every ion read and
    written once, E and B read and n, J written once per cell), the rest of
    the field phase at the minimum of 124 B per cell (previous moments in
    and out, B in and out, E out, moments read by the field advance; the
    push's 40 B per cell counted once), and the sort amortised over its
    interval (each ion's cell, offsets and velocities read once for its
    predicted key, and its fields read and written once: 20 + 2 x 28 B in
    2D, 28 + 2 x 32 B in 3D; with open faces the key is the cell alone,
    4 B)."""
    p = wl.params
    dim2 = p["ny"] == 1
    ncell = p["nx"] * p["ny"] * p["nz"]
    n = wl.n_particles
    push = push_bytes_per_launch(wl)
    field = ncell * (124 - 40)
    S = p["sort_every"]
    key = 4 if p.get("open_faces", 0) else (20 if dim2 else 28)
    sort = n * (key + 2 * (28 if dim2 else 32)) / S if S > 0 else 0.0
    return {"push": push, "field": float(field), "sort": sort, "total": push + field + sort}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def traffic_record(workload: str):
    """DRAM bytes per push launch from the committed ncu summary, valid only
    while the push kernel's source and compile-time settings are unchanged
    (a hash of both recorded with it)."""
    csrc = os.path.join(ROOT, "paper_2305_05600_gb300", "csrc")
    rec = os.path.join(ROOT, "profiles", "push_traffic.json")
    try:
        with open(rec) as f:
            d = json.load(f)
        blob = b"".join(open(os.path.join(csrc, name), "rb").read()
                        for name in ("hv_push.cu", "hv_internal.cuh"))
        h = hashlib.sha256(blob).hexdigest()[:16]
        ent = d.get(workload)
        if ent and ent.get("source_sha") == h:
            return float(ent["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_strip_rate(wl, rows: int, steps: int, threads: int = 1):
    """Time the FP64 oracle on a strip of `rows` z-rows of the workload
    (all nx columns, every ion in those rows, treated as its own periodic
    box: per-ion and per-cell costs are those of the full grid) with
    `threads` host threads.  Returns (pushes/s, ions in strip, seconds,
    per-step seconds list)."""
    import oracle as O
    O.set_threads(threads)
    try:
        return _strip_rate(O, wl, rows, steps)
    finally:
        O.set_threads(1)


def _host(a):
    """numpy copy of a species array (from the GPU for device-generated
    workloads)."""
    return a.cpu().numpy() if hasattr(a, "cpu") else a


def _strip_rate(O, wl, rows, steps):
    p = dict(wl.params)
    nx, nz = p["nx"], p["nz"]
    k0 = (nz - rows) // 2
    s = wl.species[0]
    k = s.cell // (nx * p["ny"])
    sel = (k >= k0) & (k < k0 + rows)
    cell = _host(s.cell[sel]).astype(np.int64) - k0 * nx * p["ny"]
    sp = O.Species(s.q, s.m, cell, _host(s.off[:, sel]), _host(s.v[:, sel]), _host(s.w[sel]))
    B = wl.B0[:, k0:k0 + rows].astype(np.float64).reshape(3, -1)
    g = O.make_grid(nx, p["ny"], rows, p["dx"], p["dy"], p["dz"], p["dt"], p["nsub"], p["Te"],
                    p["gamma_e"], p["eta"], p["eta_h"], p["n_floor"], p["shape"],
                    p["smooth_passes"], p.get("field_smooth_passes", 0), p.get("pe_eq", 0),
                    p.get("kappa", 0.0), p.get("ohm_model", 0), p.get("relativistic", 0),
                    p.get("c_light", 0.0))
    sim = O.Sim(g, [sp], B)
    times = []
    for i in range(steps):
        t0 = time.perf_counter()
        sim.step(1, sort_every=p["sort_every"])
        times.append(time.perf_counter() - t0)
    total = sum(times)
    return sp.n * steps / total, sp.n, total, times


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle as O
    wl = apply_overrides(make_workload(args.workload, args.shape), args)
    p = wl.params
    n_full = wl.n_particles
    cores = O.max_threads()
    # bound the whole run to ~2 minutes: rows per step from a probe
    budget = 120.0 / max(1, args.steps + args.warmup)
    probe = max(2, min(p["nz"], 2 * cores))
    _, _, t1, _ = oracle_strip_rate(wl, probe, 1, cores)
    per_row = t1 / probe
    rows = int(max(2, min(p["nz"], budget / max(per_row, 1e-6))))
    rate, n_strip, total, times = oracle_strip_rate(wl, rows, args.warmup + args.steps, cores)
    timed = times[args.warmup:]
    value = n_strip * len(timed) / sum(timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(timed) / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} ({p['nx']}x{p['ny']}x{p['nz']}, "
                               f"{n_full} ions, shape {args.shape})",
                   "sample": f"{rows}-row strip ({n_strip} ions) of the same workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{rows} of {p['nz']} z-rows, all {p['nx']} columns, "
                                   f"{n_strip} ions, periodic strip; {cores} threads "
                                   f"(private deposit grids added in thread order)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "context": {"paper_pushes_per_s_per_core": PAPER_PUSHES_PER_CORE},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import torch

    from paper_2305_05600_gb300 import hv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hv.lib()
    hv.hv_set_allocator(True)
    wl = apply_overrides(make_workload(args.workload, args.shape, seed_offset=rank), args)
    n_ions = wl.n_particles
    stream = torch.cuda.current_stream(dev)
    ctx = hv.load_workload(wl, stream=stream)

    # warm-up (the first call also runs the start-up deposit and E^0)
    for _ in range(args.warmup):
        hv.hv_step(ctx, 1)
    torch.cuda.synchronize(dev)
    if args.per_step > 0:
        per_step_profile(ctx, wl, args)
        return
    hv.hv_profile(ctx, True)
    clocks = Clocks(local, not args.no_clocks and rank == 0)
    barrier(world)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    hv.hv_step(ctx, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ck = clocks.stop()
    ms_local = ev0.elapsed_time(ev1)
    prof = hv.hv_profile_read(ctx)
    hv.hv_profile(ctx, False)
    diag = hv.hv_diag(ctx, check=False)
    ms = max_over_ranks(ms_local, world)
    total_ions = sum_over_ranks(float(n_ions), world)
    value = total_ions * args.steps / (ms * 1e-3)
    ctx.close()
    del ctx
    torch.cuda.synchronize(dev)

    # end-to-end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, wl, world, dev, stream)

    peak, peak_kind = measured_peak()
    push_ms = prof["ms_push"] / max(1, prof["n_push"])
    bytes_launch = push_bytes_per_launch(wl)
    achieved = bytes_launch / (push_ms * 1e-3) / 1e9
    traffic = traffic_record(args.workload)
    sb = step_bytes(wl)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl)

    if rank == 0:
        p = wl.params
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {p['nx']}x{p['ny']}x{p['nz']} cells, "
                                   f"dx={p['dx']}, {n_ions} ions/GPU, shape {args.shape}, "
                                   f"nsub={p['nsub']}, sort every {p['sort_every']}"
                                   + (f", {p['smooth_passes']} smoothing passes on the moments "
                                      f"and the gathered fields" if args.smooth else "")
                                   + (", electron energy equation (gamma_e 5/3, kappa 0.01)"
                                      if args.pe_eq else ""),
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (ions %.2f GB/GPU)" % (
                           n_ions * (28 if p['ny'] == 1 else 32) / 1e9)},
            "roofline": {"bound": "hbm", "kernel": "push_kernel (gather+Boris+deposit+move)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "bytes_per_launch": bytes_launch,
                         "ms_per_launch": push_ms},
            "roofline_step": {"bound": "hbm", "what": "whole step (sort amortised, push, "
                                                      "moment post, field subcycles, final Ohm)",
                              "bytes_per_step": sb["total"],
                              "bytes_split": {k: sb[k] for k in ("push", "field", "sort")},
                              "achieved": sb["total"] / (ms / args.steps * 1e-3) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": sb["total"] / (ms / args.steps * 1e-3) / 1e9 / peak,
                              "peak_kind": peak_kind},
            "phases_ms_per_step": {k: prof["ms_" + k] / max(1, prof["steps"])
                                   for k in ("sort", "push", "moments", "field", "ohm")},
            "phases_note": "sort: the sorts' own device time per step (events on the stream "
                           "each ran on); a sort issued ahead of its step overlaps the field "
                           "phase, whose time includes that overlap",
            "gpu_launches": int(prof["launches"]),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": ck,
            "diag": {k: diag[k] for k in ("W_K", "W_B", "charge", "max_divB", "err_word")},
            "context": {"paper_pushes_per_s_per_core": PAPER_PUSHES_PER_CORE},
        }
        print(json.dumps(line), flush=True)


def run_e2e(args, wl, world, dev, stream):
    """Pushes/s through the public API with ions in pinned host memory: the
    timed region holds the host->device load, every step with a
    device->host read of its diagnostics, and the final moments read."""
    import torch

    from paper_2305_05600_gb300 import hv

    if any(hasattr(s.cell, "is_cuda") for s in wl.species):
        return {"value": None, "unit": UNIT,
                "skipped": "workload generated on the GPU (no host copy of its ions)"}

    def pinned(a):
        t = torch.empty(a.shape, dtype={np.float32: torch.float32,
                                        np.int32: torch.int32}[a.dtype.type], pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    hsp = [(s.q, s.m, pinned(s.cell), pinned(s.off), pinned(s.v), pinned(s.w))
           for s in wl.species]
    p = wl.params
    nc = p["nx"] * p["ny"] * p["nz"]
    n_host = np.zeros((p["nz"], p["ny"], p["nx"]), np.float32)
    J_host = np.zeros((3, p["nz"], p["ny"], p["nx"]), np.float32)
    steps = max(1, args.steps)  # as many steps as the device-timed loop
    ctx = hv.hv_init_grid(p, wl.B0, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ev[0].record(stream)
    for i, (q, m, c, o, v, w) in enumerate(hsp):
        hv.hv_load_ions(ctx, i, q, m, c, o, v, w)
        if wl.reserve > 0.0:
            hv.hv_reserve_ions(ctx, i, int(wl.reserve * c.shape[0]) + 1024)
    for s_idx, face, n_b, u_b, T_b, w_b in wl.inject:
        hv.hv_set_injection(ctx, s_idx, face, n_b, u_b, T_b, w_b)
    ev[1].record(stream)
    # every step's diagnostics are read on the host, one step behind, so that
    # the next step is already queued while the host waits for them
    for i in range(steps):
        hv.hv_step(ctx, 1)
        hv.hv_diag_async(ctx)
        if i > 0:
            hv.hv_diag_wait(ctx)
    hv.hv_diag_wait(ctx)
    hv.hv_moments(ctx, n_host, J_host, None, None)
    ev[2].record(stream)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    load_ms = ev[0].elapsed_time(ev[1])
    steps_ms = ev[1].elapsed_time(ev[2])
    barrier(world)
    ctx.close()
    dt = max_over_ranks(dt, world)
    n_ions = sum_over_ranks(float(wl.n_particles), world)
    h2d = sum(a.nbytes for s in hsp for a in s[2:]) / steps
    d2h = 80 + (n_host.nbytes + J_host.nbytes) / steps
    return {"value": n_ions * steps / dt, "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "note": "load amortised over the steps; every step's diagnostics read on the "
                    "host (hv_diag_async / hv_diag_wait, one step behind)",
            "device_ms": {"load": round(load_ms, 3), "steps_with_startup_and_reads":
                          round(steps_ms, 3)}}


def cpu_baseline(wl):
    """The FP64 oracle on the host's cores (all of them, and one thread for
    comparison), each on a strip of the workload sized to ~8 s of work."""
    import oracle as O
    nz = wl.params["nz"]
    out = {}
    for label, threads in (("single", 1), ("all", O.max_threads())):
        probe = max(2, min(nz, 2 * threads))
        _, _, t2, _ = oracle_strip_rate(wl, probe, 1, threads)
        rows = int(max(2, min(nz, 8.0 / max(t2 / probe, 1e-6))))
        rate, n_strip, total, _ = oracle_strip_rate(wl, rows, 1, threads)
        out[label] = {"value": rate, "threads": threads,
                      "sample": f"one step of a {rows}-of-{nz}-row strip ({n_strip} ions, all "
                                f"{wl.params['nx']} columns) of the same workload, periodic "
                                f"({total:.1f} s)"}
    a = out["all"]
    return {"value": a["value"], "unit": UNIT, "cores": a["threads"], "kind": "oracle",
            "sample": a["sample"] + f", {a['threads']} threads (private deposit grids added "
                                    f"in thread order)",
            "single_thread": {"value": out["single"]["value"], "unit": UNIT, "cores": 1,
                              "sample": out["single"]["sample"]}}


def per_step_profile(ctx, wl, args):
    """Push time of single steps against the steps since the last sort
    (device time of the push phase, events on its stream), averaged over
    the profiled steps with the same count; one JSON line."""
    from paper_2305_05600_gb300 import hv
    S = wl.params["sort_every"]
    step0 = hv.hv_query(ctx)["step"]
    times = {}
    for _ in range(args.per_step):
        since = (hv.hv_query(ctx)["step"] % S) if S > 0 else -1
        hv.hv_profile(ctx, True)
        hv.hv_step(ctx, 1)
        p = hv.hv_profile_read(ctx)
        times.setdefault(since, []).append(p["ms_push"] / max(1, p["n_push"]))
    hv.hv_profile(ctx, False)
    print(json.dumps({"workload": args.workload, "sort_every": S, "first_step": step0,
                      "steps": args.per_step,
                      "push_ms_by_steps_since_sort": {str(k): round(sum(v) / len(v), 4)
                                                      for k, v in sorted(times.items())}}))


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
