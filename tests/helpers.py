"""Shared test helpers: convert seeded workloads into oracle objects and
compare particle states by physical position."""
import numpy as np

import oracle as O


def oracle_grid(p, **over):
    q = dict(p)
    q.update(over)
    return O.make_grid(q["nx"], q["ny"], q["nz"], q["dx"], q["dy"], q["dz"], q["dt"],
                       q["nsub"], q["Te"], q["gamma_e"], q["eta"], q["eta_h"], q["n_floor"],
                       q["shape"], q["smooth_passes"], q.get("field_smooth_passes", 0),
                       q.get("pe_eq", 0), q.get("kappa", 0.0), q.get("ohm_model", 0),
                       q.get("relativistic", 0), q.get("c_light", 0.0))


def oracle_species(wl):
    return [O.Species(s.q, s.m, s.cell.astype(np.int64), s.off.astype(np.float64),
                      s.v.astype(np.float64), s.w.astype(np.float64)) for s in wl.species]


def oracle_sim(wl, **over):
    g = oracle_grid(wl.params, **over)
    return O.Sim(g, oracle_species(wl), wl.B0.astype(np.float64).reshape(3, -1))


def phys_pos(p, cell, off):
    """Physical coordinates (3, n) of particles from cell + relative offsets."""
    cell = np.asarray(cell, dtype=np.int64)
    nx, ny = p["nx"], p["ny"]
    idx = np.stack([cell % nx, (cell // nx) % ny, cell // (nx * ny)])
    dl = np.array([p["dx"], p["dy"], p["dz"]])[:, None]
    return (idx + 0.5 + 0.5 * np.asarray(off, dtype=np.float64)) * dl


def periodic_delta(p, a, b):
    """Minimum-image difference a - b of physical coordinates (3, n)."""
    L = np.array([p["nx"] * p["dx"], p["ny"] * p["dy"], p["nz"] * p["dz"]])[:, None]
    d = a - b
    return d - L * np.round(d / L)
