"""Shared test helpers: convert seeded workloads into oracle objects and
compare particle states by physical position."""
import numpy as np

import oracle as O


def oracle_grid(p, B0ext=None, **over):
    q = dict(p)
    q.update(over)
    return O.make_grid(q["nx"], q["ny"], q["nz"], q["dx"], q["dy"], q["dz"], q["dt"],
                       q["nsub"], q["Te"], q["gamma_e"], q["eta"], q["eta_h"], q["n_floor"],
                       q["shape"], q["smooth_passes"], q.get("field_smooth_passes", 0),
                       q.get("pe_eq", 0), q.get("kappa", 0.0), q.get("ohm_model", 0),
                       q.get("relativistic", 0), q.get("c_light", 0.0),
                       open_axes=[(int(q.get("open_faces", 0)) >> a) & 1 for a in range(3)],
                       B0ext=B0ext)


def oracle_species(wl):
    return [O.Species(s.q, s.m, s.cell.astype(np.int64), s.off.astype(np.float64),
                      s.v.astype(np.float64), s.w.astype(np.float64)) for s in wl.species]


def oracle_sim(wl, B0ext=None, inject=None, seed=0, **over):
    g = oracle_grid(wl.params, B0ext=B0ext, **over)
    return O.Sim(g, oracle_species(wl), wl.B0.astype(np.float64).reshape(3, -1), inject=inject,
                 seed=seed)


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


def check_diagnostics(p, d, sim, B_gpu, B0ext=None):
    """The FP64 diagnostics of a GPU step against the oracle's step.

    * charge within 1e-6 and W_K within 1e-5 relative, W_B within 1e-6;
    * each momentum component P_a = sum m w v_a: the GPU sums FP32 products
      (Kahan-compensated per lane, FP64 across lanes), so its error is a few
      FP32 roundings of the summed magnitudes; the bound is 1e-6 of
      sum m w |v_a| (P itself may be near zero by symmetry);
    * max |div B|: the GPU evaluates the centred divergence (Eq. 12) of its
      own B in FP32 (FP64 is kept for the conservation sums): it must equal
      the oracle's FP64 divergence of the GPU's B to within the FP32
      rounding of that stencil (each difference, product and sum rounded
      once: 5 * 2^-24 * sum_a max|B_a| / Delta_a), and differ from the
      oracle's own value by at most that plus the divergence the FP32
      difference of the two B fields can carry, sum_a max|dB_a| / Delta_a
      (div is linear and its stencil is (B[+1] - B[-1]) / (2 Delta))."""
    od = sim.diags[-1]
    assert abs(d["charge"] - od["charge"]) < 1e-6 * abs(od["charge"])
    assert abs(d["W_K"] - od["W_K"]) < 1e-5 * od["W_K"]
    assert abs(d["W_B"] - od["W_B"]) < 1e-6 * od["W_B"]
    absP = np.zeros(3)
    for s in sim.species:
        absP += np.sum(s.m * s.w * np.abs(s.v), axis=1)
    for a in range(3):
        assert abs(d["P"][a] - od["P"][a]) <= 1e-6 * absP[a], (a, d["P"][a], od["P"][a], absP[a])
    B_gpu = np.asarray(B_gpu, np.float64).reshape(3, -1)
    dl = (p["dx"], p["dy"], p["dz"])
    nn = (p["nx"], p["ny"], p["nz"])
    slack = 0.0
    if B0ext is None:
        g = oracle_grid(p)
        md_own = O.max_div(g, B_gpu)  # periodic neighbours, or open-face ghost copies
        fp32 = sum(5.0 * 2.0 ** -24 * np.abs(B_gpu[a]).max() / dl[a] for a in range(3)
                   if nn[a] > 1)
        assert abs(d["max_divB"] - md_own) <= fp32, (d["max_divB"], md_own, fp32)
        slack = fp32
    else:
        # hv_moments reports B0 + B1 rounded to FP32; the divergence is of B1
        B_gpu = B_gpu - np.asarray(B0ext, np.float64).reshape(3, -1)
        bt = np.abs(B_gpu) + np.abs(np.asarray(B0ext, np.float64).reshape(3, -1))
        slack = sum((2.0 ** -23 + 5.0 * 2.0 ** -24) * bt[a].max() / dl[a]
                    for a in range(3) if nn[a] > 1)
    dB = np.abs(B_gpu - sim.B)
    bound = sum(dB[a].max() / dl[a] for a in range(3) if nn[a] > 1) + slack
    assert abs(d["max_divB"] - od["max_divB"]) <= bound + 1e-12, (d["max_divB"], od["max_divB"],
                                                                  bound)
