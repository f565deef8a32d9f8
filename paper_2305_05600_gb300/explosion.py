"""Expanding-cloud check of particle shape and smoothing (Sec. 3.2, the
astrophysical explosion).

The paper runs a debris cloud expanding at 15 v_A into a magnetised
background on a deliberately coarse grid (1000 d_i in 512 cells) twice: with
NGP weights the shock front stays coherent; with QS weights and 10 passes
of moment and field smoothing it breaks into filaments, and the leading
filament outruns the rest of the front.  This module runs both cases with
libhv (`inputs.explosion2d`, row f1 of the build: the smoothing of the
gathered fields included) and measures the front along rays from the cloud
centre, in two sectors of +-20 degrees: across B0 (around the z axis) and
along B0 (around the x axis).  On each ray the total density, box-averaged
over 3x3 cells (analysis only), is sampled every half cell:

  * layers: separate compressed shells, counted with hysteresis (a layer
    starts where the density rises above 1.5 n0 and ends where it falls
    below 1.2 n0);
  * r_lead: the outermost radius above 1.5 n0 (the leading edge);
  * r_peak: the radius of the density maximum.

The sector values are the mean layer count, the fraction of rays with two
or more layers and the medians of r_lead and r_peak.

    python -m paper_2305_05600_gb300.explosion --out explosion.json
    python -m paper_2305_05600_gb300.explosion --summarize explosion.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import hv
from . import inputs as I

CASES = {"ngp": ("ngp", 0), "qs_smooth10": ("qs", 10)}
SECTORS = {"across_B0": 0.5 * math.pi, "along_B0": 0.0}


def box3(n: np.ndarray) -> np.ndarray:
    """3x3 periodic box average of a [nz][nx] array."""
    s = np.zeros_like(n, dtype=np.float64)
    for dz in (-1, 0, 1):
        for dx in (-1, 0, 1):
            s += np.roll(np.roll(n, dz, axis=0), dx, axis=1)
    return s / 9.0


def sample_rays(n: np.ndarray, dx: float, th: np.ndarray, r: np.ndarray,
                center=None) -> np.ndarray:
    """The 3x3-averaged density [nz][nx] sampled along rays from `center`
    (physical coordinates, default the box centre) at angles th (from +x
    towards +z) and radii r, bilinear on the cell centres: [len(th)][len(r)]."""
    nz, nx = n.shape
    ns = box3(np.asarray(n, np.float64))
    xc, zc = (0.5 * nx * dx, 0.5 * nz * dx) if center is None else center
    X = (xc + r[None, :] * np.cos(th)[:, None]) / dx - 0.5
    Z = (zc + r[None, :] * np.sin(th)[:, None]) / dx - 0.5
    i0 = np.floor(X).astype(np.int64)
    k0 = np.floor(Z).astype(np.int64)
    fx, fz = X - i0, Z - k0
    i0 %= nx
    k0 %= nz
    i1, k1 = (i0 + 1) % nx, (k0 + 1) % nz
    return ((1 - fx) * (1 - fz) * ns[k0, i0] + fx * (1 - fz) * ns[k0, i1] +
            (1 - fx) * fz * ns[k1, i0] + fx * fz * ns[k1, i1])


def layer_count(p: np.ndarray, hi: float = 1.5, lo: float = 1.2) -> int:
    """Separate shells along a radial profile: rises above `hi` that follow
    a fall below `lo` (or the start)."""
    count, inside = 0, False
    for v in p:
        if not inside and v > hi:
            count += 1
            inside = True
        elif inside and v < lo:
            inside = False
    return count


def sector_metrics(n: np.ndarray, dx: float, angle: float, half_width: float = math.radians(20),
                   nray: int = 81, hi: float = 1.5, lo: float = 1.2) -> dict:
    """Layer count, leading edge and peak radius over the rays of the two
    opposite sectors of +-half_width about `angle` (see the module text)."""
    nz, nx = n.shape
    a = np.linspace(-half_width, half_width, nray)
    th = np.concatenate([angle + a, angle + math.pi + a])
    r = 0.5 * dx * np.arange(1, int(0.98 * min(nx, nz)))
    P = sample_rays(n, dx, th, r)
    layers = np.array([layer_count(p, hi, lo) for p in P])
    above = P > hi
    lead = np.array([r[np.nonzero(q)[0].max()] if q.any() else 0.0 for q in above])
    peak = r[np.argmax(P, axis=1)]
    return {"layers": float(layers.mean()), "multi": float((layers >= 2).mean()),
            "r_lead": float(np.median(lead)), "r_peak": float(np.median(peak)),
            "n_max": float(np.median(P.max(axis=1)))}


def run_case(shape: str, passes: int, steps: int, every: int, snap_at=(), **kw) -> dict:
    wl = I.explosion2d(shape=shape, smooth_passes=passes, **kw)
    p = wl.params
    ctx = hv.load_workload(wl)
    del wl
    hv.hv_profile(ctx, True)
    hist, snaps, failed = [], {}, None
    t0 = time.perf_counter()
    try:
        for s in range(0, steps + 1, every):
            if s > 0:
                hv.hv_step(ctx, every)
            n = hv.hv_moments(ctx)["n"].reshape(p["nz"], p["nx"])
            m = {"t": s * p["dt"], "step": s}
            for name, ang in SECTORS.items():
                m[name] = sector_metrics(n, p["dx"], ang)
            hist.append(m)
            if s in snap_at:
                snaps[s] = n.copy()
    except hv.HVError as e:
        failed = {"step": s, "error": str(e)}
    wall = time.perf_counter() - t0
    prof = hv.hv_profile_read(ctx)
    ctx.close()
    gpu_ms = sum(prof["ms_" + k] for k in ("sort", "push", "moments", "field", "ohm"))
    return {"shape": shape, "passes": passes, "history": hist, "density": snaps,
            "ms_per_step": gpu_ms / max(1, prof["steps"]), "wall_s": wall, "failed": failed,
            "params": {k: p[k] for k in ("nx", "nz", "dx", "dt", "nsub", "eta", "eta_h",
                                         "n_floor")}}


def summarize(res: dict) -> str:
    cases = res["cases"]
    lines = ["| t | sector | " + " | ".join(f"{c}: layers, >=2, r_lead, r_peak" for c in cases)
             + " | r_lead ratio |", "|---:|---|" + "---|" * len(cases) + "---:|"]
    names = list(cases)
    hists = [{h["step"]: h for h in cases[c]["history"]} for c in names]
    for step in sorted(hists[0]):
        if step == 0 or step % res["report_every"] or any(step not in h for h in hists):
            continue
        for sec in SECTORS:
            cells = []
            for h in hists:
                m = h[step][sec]
                cells.append(f"{m['layers']:.2f}, {m['multi']:.2f}, {m['r_lead']:.0f}, "
                             f"{m['r_peak']:.0f}")
            ratio = hists[-1][step][sec]["r_lead"] / max(hists[0][step][sec]["r_lead"], 1e-9)
            lines.append(f"| {hists[0][step]['t']:.0f} | {sec} | " + " | ".join(cells)
                         + f" | {ratio:.3f} |")
    for c in names:
        lines.append(f"\n{c}: {cases[c]['ms_per_step']:.3f} ms per step on the GPU"
                     + (f"; stopped: {cases[c]['failed']}" if cases[c]["failed"] else ""))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="explosion.json")
    ap.add_argument("--npz", default=None, help="also save the density snapshots here")
    ap.add_argument("--summarize", default=None)
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ppc", type=int, default=200)
    ap.add_argument("--n-debris", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--report-every", type=int, default=500)
    a = ap.parse_args()
    if a.summarize:
        print(summarize(json.load(open(a.summarize))))
        return
    hv.lib()
    hv.hv_set_allocator(True)
    scale = a.nx / 512
    kw = dict(nx=a.nx, nz=a.nx, length=1000.0 * scale, ppc=a.ppc, n_debris=a.n_debris,
              r_m=150.0 * scale)
    snap_at = set(range(0, a.steps + 1, a.report_every))
    res = {"config": dict(kw, steps=a.steps), "report_every": a.report_every, "cases": {}}
    dens = {}
    for name, (shape, passes) in CASES.items():
        c = run_case(shape, passes, a.steps, a.every, snap_at=snap_at, **kw)
        for st, n in c.pop("density").items():
            dens[f"{name}_{st}"] = n.astype(np.float32)
        res["cases"][name] = c
        json.dump(res, open(a.out, "w"))
    if a.npz:
        np.savez_compressed(a.npz, **dens)
    print(summarize(res))


if __name__ == "__main__":
    main()
