"""Resistive hose check of the kinetic-electron beam model (App. A).

A relativistic electron beam (gamma = 2.96, about 1 MeV) with a sech^2
current channel in a resistive background (E = eta (curl B - J_k)) is
unstable to the resistive hose: the channel kinks, faster for larger
resistivity, and stays put without resistivity.  This module runs
`inputs.ebeam2d` (80 x 20 d_e on 640 x 320 cells, periodic) for several eta
with libhv and measures, from the deposited electron density, the channel
centroid zbar(x) of every column and its RMS displacement over x (the kink
amplitude) and the RMS channel width.

    python -m paper_2305_05600_gb300.hose --out hose.json
    python -m paper_2305_05600_gb300.hose --summarize hose.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import hv
from . import inputs as I


def channel(n: np.ndarray, dz: float) -> tuple[float, float]:
    """Kink amplitude (RMS over x of the column centroids about their mean)
    and RMS width of a channel density |n| [nz][nx] centred in z."""
    a = np.abs(np.asarray(n, np.float64))
    nz = a.shape[0]
    z = (np.arange(nz) + 0.5) * dz
    mass = a.sum(axis=0)
    zbar = (a * z[:, None]).sum(axis=0) / mass
    kink = float(np.sqrt(np.mean((zbar - zbar.mean()) ** 2)))
    width = float(np.sqrt((a * (z[:, None] - zbar[None, :]) ** 2).sum() / a.sum()))
    return kink, width


def run_case(eta: float, steps: int, every: int, **kw) -> dict:
    wl = I.ebeam2d(eta=eta, **kw)
    p = wl.params
    ctx = hv.load_workload(wl)
    del wl
    hv.hv_profile(ctx, True)
    hist, failed = [], None
    t0 = time.perf_counter()
    try:
        for s in range(0, steps + 1, every):
            if s > 0:
                hv.hv_step(ctx, every)
            n = hv.hv_moments(ctx)["n"].reshape(p["nz"], p["nx"])
            kink, width = channel(n, p["dz"])
            hist.append({"step": s, "t": s * p["dt"], "kink": kink, "width": width})
    except hv.HVError as e:
        failed = {"step": s, "error": str(e)}
    wall = time.perf_counter() - t0
    prof = hv.hv_profile_read(ctx)
    ctx.close()
    gpu_ms = sum(prof["ms_" + k] for k in ("sort", "push", "moments", "field", "ohm"))
    return {"eta": eta, "history": hist, "ms_per_step": gpu_ms / max(1, prof["steps"]),
            "wall_s": wall, "failed": failed}


def summarize(res: dict) -> str:
    cases = res["cases"]
    names = list(cases)
    lines = ["| t | " + " | ".join(f"eta={cases[c]['eta']:g}: kink, width" for c in names) + " |",
             "|---:|" + "---|" * len(names)]
    hists = [{h["step"]: h for h in cases[c]["history"]} for c in names]
    for step in sorted(hists[0]):
        if step % res["report_every"] or any(step not in h for h in hists):
            continue
        cells = [f"{h[step]['kink']:.4f}, {h[step]['width']:.3f}" for h in hists]
        lines.append(f"| {hists[0][step]['t']:.0f} | " + " | ".join(cells) + " |")
    for c in names:
        lines.append(f"\neta={cases[c]['eta']:g}: {cases[c]['ms_per_step']:.3f} ms per step on the "
                     "GPU" + (f"; stopped: {cases[c]['failed']}" if cases[c]["failed"] else ""))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="hose.json")
    ap.add_argument("--summarize", default=None)
    ap.add_argument("--etas", default="0,0.01,0.1")
    ap.add_argument("--steps", type=int, default=7500)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--report-every", type=int, default=1250)
    ap.add_argument("--ppc", type=int, default=64)
    a = ap.parse_args()
    if a.summarize:
        print(summarize(json.load(open(a.summarize))))
        return
    hv.lib()
    hv.hv_set_allocator(True)
    res = {"config": {"steps": a.steps, "ppc": a.ppc}, "report_every": a.report_every,
           "cases": {}}
    for eta in (float(x) for x in a.etas.split(",")):
        res["cases"][f"eta_{eta:g}"] = run_case(eta, a.steps, a.every, ppc=a.ppc)
        json.dump(res, open(a.out, "w"))
    print(summarize(res))


if __name__ == "__main__":
    main()
