"""Seeded synthetic workloads for the hybrid PIC ion loop.

This module only builds inputs: grid parameters, the initial magnetic field
and ion macro-particles.  It contains none of the method's arithmetic (no
push, shape, deposit or field solve).  Both the CUDA library and the CPU
oracle consume exactly the arrays produced here (FP32 particles and FP32 B;
the oracle upcasts them), so both sides start from identical states.

Units are normalised Alfvenic units (e = m_p = mu_0 = n_0 = B_0 = 1, lengths
in d_i, time in 1/Omega_ci).  2D runs are x-z planes with ny = 1.

Workloads (sizes as named; ``scaled`` variants keep the profile on a smaller
grid for parity tests):

* ``alfven2d``   periodic uniform plasma 64x64, dx = 0.5, 64 ppc, beta_i =
  beta_e = 0.5, B0 = x^ plus an Alfven wave dB_y = 0.01 sin(k x), k = 2 pi/Lx,
  with the matching ion drift, dt = 0.01, 10 field subcycles.
* ``harris2d``   double periodic Harris sheet 1024x512, dx = 0.25, 100 ppc,
  half-width 1, background 0.2, Ti/Te = 5, 0.1 B0 X-point perturbation,
  eta = 1e-3, eta_H = 1e-4, density floor 0.05, dt = 0.02, 10 subcycles.
* ``beam3d``     periodic ion-ion beam 256x128x128, dx = 0.5, 56 core + 8 beam
  ions per cell (5% beam density at 10 v_A along B0), beta_i = 0.1.
* ``harris3d``   the Harris sheet in 3D (uniform in y) with guide field
  B_y = 0.1, 32 ppc.
* ``whistler1d`` quasi-1D 128x1x1 cold plasma, dx = 0.25, 256 ppc, one
  circularly mixed Alfven/whistler mode for the dispersion measurement.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SpeciesInput:
    q: float
    m: float
    cell: np.ndarray  # int32 [n]
    off: np.ndarray   # float32 [3][n], relative coordinates in [-1, 1)
    v: np.ndarray     # float32 [3][n], v^{-1/2}
    w: np.ndarray     # float32 [n]

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])


@dataclass
class Workload:
    name: str
    params: dict
    B0: np.ndarray                      # float32 [3][nz][ny][nx]
    species: list = field(default_factory=list)
    steps: int = 1
    notes: str = ""
    # open faces: (species, face, n, u, T, w) injected every step, and the
    # particle slots to reserve per species as a multiple of its ions
    inject: list = field(default_factory=list)
    reserve: float = 0.0

    @property
    def n_particles(self) -> int:
        return sum(s.n for s in self.species)

    @property
    def ncell(self) -> int:
        p = self.params
        return p["nx"] * p["ny"] * p["nz"]


def base_params(nx, ny, nz, dx, dy, dz, dt, nsub, Te, eta=0.0, eta_h=0.0, n_floor=0.05,
                shape="qs", smooth_passes=0, gamma_e=1.0, sort_every=20, field_smooth_passes=0,
                pe_eq=0, kappa=0.0, ohm_model=0, relativistic=0, c_light=0.0):
    return dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy if ny > 1 else 1.0, dz=dz, dt=dt,
                nsub=nsub, Te=Te, gamma_e=gamma_e, eta=eta, eta_h=eta_h, n_floor=n_floor,
                shape=shape, smooth_passes=smooth_passes, sort_every=sort_every,
                field_smooth_passes=field_smooth_passes, pe_eq=pe_eq, kappa=kappa,
                ohm_model=ohm_model, relativistic=relativistic, c_light=c_light)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _box_muller(rng: np.random.Generator, shape) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniforms."""
    u1 = 1.0 - rng.random(shape)  # (0, 1]
    u2 = rng.random(shape)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def cell_centres(p):
    """Cell-centre coordinates (x, y, z) as 1D arrays."""
    x = (np.arange(p["nx"]) + 0.5) * p["dx"]
    y = (np.arange(p["ny"]) + 0.5) * p["dy"]
    z = (np.arange(p["nz"]) + 0.5) * p["dz"]
    return x, y, z


def _curl_of_vector_potential(p, Ax=None, Ay=None, Az=None):
    """B = curl A with the centred periodic difference, so that the initial
    field has zero discrete divergence.  A* are [nz][ny][nx] float64."""
    shape = (p["nz"], p["ny"], p["nx"])
    zero = np.zeros(shape)
    Ax = zero if Ax is None else Ax
    Ay = zero if Ay is None else Ay
    Az = zero if Az is None else Az

    def d(f, axis, h):
        return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * h)

    ax_x, ax_y, ax_z = 2, 1, 0
    Bx = d(Az, ax_y, p["dy"]) - d(Ay, ax_z, p["dz"])
    By = d(Ax, ax_z, p["dz"]) - d(Az, ax_x, p["dx"])
    Bz = d(Ay, ax_x, p["dx"]) - d(Ax, ax_y, p["dy"])
    return np.stack([Bx, By, Bz])


def load_cells(p, ppc_of_cell, rng, dims3):
    """Cell-major particle placement: ``ppc_of_cell`` [ncell] particles in each
    cell, relative coordinates uniform in [-1, 1) along each axis with more
    than one cell (0 along a single-cell axis)."""
    counts = np.asarray(ppc_of_cell, dtype=np.int64)
    cell = np.repeat(np.arange(counts.shape[0], dtype=np.int64), counts)
    n = cell.shape[0]
    off = np.zeros((3, n))
    for a, na in enumerate(dims3):
        if na > 1:
            off[a] = rng.uniform(-1.0, 1.0, n)
    return cell, off


def positions(p, cell, off):
    """Physical positions of particles (x, y, z), each [n] float64."""
    nx, ny = p["nx"], p["ny"]
    i = cell % nx
    j = (cell // nx) % ny
    k = cell // (nx * ny)
    x = (i + 0.5 + 0.5 * off[0]) * p["dx"]
    y = (j + 0.5 + 0.5 * off[1]) * p["dy"]
    z = (k + 0.5 + 0.5 * off[2]) * p["dz"]
    return x, y, z


def _finish(cell, off, v, w, q=1.0, m=1.0) -> SpeciesInput:
    off32 = off.astype(np.float32)
    # rounding to float32 can produce exactly +1, which lies outside [-1, 1):
    # pull such coordinates to the largest float32 below 1 (same cell).
    off32 = np.where(off32 >= np.float32(1.0), np.nextafter(np.float32(1.0), np.float32(0.0)),
                     off32).astype(np.float32)
    return SpeciesInput(q=q, m=m, cell=cell.astype(np.int32), off=np.ascontiguousarray(off32),
                        v=np.ascontiguousarray(v.astype(np.float32)),
                        w=np.ascontiguousarray(w.astype(np.float32)))


def distinct_weights(w: np.ndarray) -> np.ndarray:
    """The float32 weights moved up by the fewest ulps that make every value
    distinct (ties broken in index order).  The library reorders ions as it
    steps but copies each weight bit for bit, so a caller that loads
    distinct weights can identify every ion afterwards."""
    w = np.asarray(w, np.float32).copy()
    order = np.argsort(w, kind="stable")
    ws = w[order]
    up = np.float32(np.inf)
    for k in range(1, ws.shape[0]):
        if ws[k] <= ws[k - 1]:
            ws[k] = np.nextafter(ws[k - 1], up)
    w[order] = ws
    return w


def with_distinct_weights(wl: "Workload") -> "Workload":
    """The workload with distinct_weights applied across all its species."""
    sizes = [s.n for s in wl.species]
    allw = distinct_weights(np.concatenate([s.w for s in wl.species]))
    o = 0
    for k, s in enumerate(wl.species):
        wl.species[k] = SpeciesInput(s.q, s.m, s.cell, s.off, s.v,
                                     np.ascontiguousarray(allw[o:o + sizes[k]]))
        o += sizes[k]
    return wl


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def alfven2d(nx=64, nz=64, ppc=64, dx=0.5, seed=0, steps=200, shape="qs", sort_every=20,
             amp=0.01) -> Workload:
    """Uniform periodic plasma with one Alfven wave (beta_i = beta_e = 0.5)."""
    p = base_params(nx, 1, nz, dx, 1.0, dx, 0.01, 10, Te=0.25, shape=shape,
                    sort_every=sort_every)
    rng = _rng(seed)
    Lx = nx * dx
    k = 2.0 * np.pi / Lx
    x, _, _ = cell_centres(p)
    # B0 = x^ + dB_y sin(kx) built from A_z = amp cos(kx)/k (B_y = -dA_z/dx)
    Az = np.broadcast_to((amp * np.cos(k * x) / k)[None, None, :], (nz, 1, nx)).copy()
    B = _curl_of_vector_potential(p, Az=Az)
    B[0] += 1.0
    ncell = nx * nz
    cell, off = load_cells(p, np.full(ncell, ppc), rng, (nx, 1, nz))
    n = cell.shape[0]
    Ti = 0.25
    v = np.sqrt(Ti) * _box_muller(rng, (3, n))
    xp, _, _ = positions(p, cell, off)
    v[1] += -amp * np.sin(k * xp)
    w = np.full(n, 1.0 * dx * dx / ppc)
    return Workload("alfven2d", p, B.astype(np.float32), [_finish(cell, off, v, w)], steps,
                    notes=f"{nx}x{nz} cells, {ppc} ppc, dx={dx}, seed={seed}")


def harris_profile(z, Lz, lam=1.0, nb=0.2):
    z1, z2 = 0.25 * Lz, 0.75 * Lz
    Bx = np.tanh((z - z1) / lam) - np.tanh((z - z2) / lam) - 1.0
    ns1 = 1.0 / np.cosh((z - z1) / lam) ** 2
    ns2 = 1.0 / np.cosh((z - z2) / lam) ** 2
    return Bx, ns1, ns2, nb


def harris(nx=1024, ny=1, nz=512, ppc=100, dx=0.25, seed=1000, steps=2000, shape="qs",
           guide=0.0, sort_every=20, lam=1.0, nb=0.2, pert=0.1, dt=0.02, nsub=10,
           smooth_passes=0, name=None) -> Workload:
    """Double periodic Harris sheet (sheets at Lz/4 and 3Lz/4) with a localised
    X-point perturbation on the upper sheet.  T_i + T_e = 0.5, T_i/T_e = 5.
    Sheet ions drift +-U_y = 2 T_i / lam; background ions are at rest."""
    p = base_params(nx, ny, nz, dx, dx, dx, dt, nsub, Te=1.0 / 12.0, eta=1e-3, eta_h=1e-4,
                    n_floor=0.05, shape=shape, smooth_passes=smooth_passes,
                    sort_every=sort_every)
    rng = _rng(seed)
    Ti = 5.0 / 12.0
    Lx, Lz = nx * dx, nz * dx
    x, y, z = cell_centres(p)
    Bx_z, ns1_z, ns2_z, _ = harris_profile(z, Lz, lam, nb)
    # X-point perturbation: A_y = A0 exp(-r^2 / (2 w^2)), w = 2 lam, centred on
    # the upper sheet; A0 gives a peak |dB| of `pert`.
    wdt = 2.0 * lam
    A0 = pert * wdt * math.exp(0.5)
    X, Z = np.meshgrid(x, z)  # [nz][nx]
    Ay2 = A0 * np.exp(-((X - 0.5 * Lx) ** 2 + (Z - 0.75 * Lz) ** 2) / (2.0 * wdt ** 2))
    Ay = np.broadcast_to(Ay2[:, None, :], (nz, ny, nx)).copy()
    B = _curl_of_vector_potential(p, Ay=Ay)
    B[0] += Bx_z[:, None, None]
    B[1] += guide
    ncell = nx * ny * nz
    # per-cell split of ppc between the two sheets and the background
    kz = np.arange(ncell) // (nx * ny)
    n_tot = ns1_z + ns2_z + nb
    c1 = np.floor(ppc * ns1_z / n_tot + 0.5).astype(np.int64)
    c2 = np.floor(ppc * ns2_z / n_tot + 0.5).astype(np.int64)
    cb = ppc - c1 - c2
    vc = dx * p["dy"] * dx
    species_parts = []
    U = 2.0 * Ti / lam
    for counts_z, dens_z, drift in ((c1, ns1_z, U), (c2, ns2_z, -U), (cb, np.full(nz, nb), 0.0)):
        counts = counts_z[kz]
        cell, off = load_cells(p, counts, rng, (nx, ny, nz))
        nn = cell.shape[0]
        v = np.sqrt(Ti) * _box_muller(rng, (3, nn))
        v[1] += drift
        kk = cell // (nx * ny)
        w = dens_z[kk] * vc / np.maximum(counts_z[kk], 1)
        species_parts.append((cell, off, v, w))
    # interleave the three populations in cell order (one species, q = m = 1)
    cell = np.concatenate([s[0] for s in species_parts])
    order = np.argsort(cell, kind="stable")
    cell = cell[order]
    off = np.concatenate([s[1] for s in species_parts], axis=1)[:, order]
    v = np.concatenate([s[2] for s in species_parts], axis=1)[:, order]
    w = np.concatenate([s[3] for s in species_parts])[order]
    nm = name or ("harris2d" if ny == 1 else "harris3d")
    return Workload(nm, p, B.astype(np.float32), [_finish(cell, off, v, w)], steps,
                    notes=f"{nx}x{ny}x{nz} cells, {ppc} ppc, dx={dx}, guide={guide}, seed={seed}")


def harris2d(**kw) -> Workload:
    return harris(**kw)


def harris3d(nx=512, ny=256, nz=256, ppc=32, dx=0.5, seed=3000, steps=1000, **kw) -> Workload:
    return harris(nx=nx, ny=ny, nz=nz, ppc=ppc, dx=dx, seed=seed, steps=steps, guide=0.1,
                  dt=kw.pop("dt", 0.02), **kw)


def beam3d(nx=256, ny=128, nz=128, n_core=56, n_beam=8, dx=0.5, seed=2000, steps=1000,
           shape="qs", sort_every=20, dt=0.01, nsub=10) -> Workload:
    """Core protons plus a 5% beam drifting at 10 v_A along B0 = x^;
    beta_i = 0.1 (T_i = 0.05 for both), isothermal electrons with T_e = 0.05."""
    p = base_params(nx, ny, nz, dx, dx, dx, dt, nsub, Te=0.05, shape=shape,
                    sort_every=sort_every)
    rng = _rng(seed)
    ncell = nx * ny * nz
    B = np.zeros((3, nz, ny, nx))
    B[0] = 1.0
    vc = dx * dx * dx
    parts = []
    for cnt, dens, drift in ((n_core, 0.95, 0.0), (n_beam, 0.05, 10.0)):
        cell, off = load_cells(p, np.full(ncell, cnt), rng, (nx, ny, nz))
        nn = cell.shape[0]
        v = math.sqrt(0.05) * _box_muller(rng, (3, nn))
        v[0] += drift
        w = np.full(nn, dens * vc / cnt)
        parts.append((cell, off, v, w))
    cell = np.concatenate([s[0] for s in parts])
    order = np.argsort(cell, kind="stable")
    cell = cell[order]
    off = np.concatenate([s[1] for s in parts], axis=1)[:, order]
    v = np.concatenate([s[2] for s in parts], axis=1)[:, order]
    w = np.concatenate([s[3] for s in parts])[order]
    return Workload("beam3d", p, B.astype(np.float32), [_finish(cell, off, v, w)], steps,
                    notes=f"{nx}x{ny}x{nz} cells, {n_core}+{n_beam} ppc, seed={seed}")


def whistler1d(nx=128, ppc=256, dx=0.25, dt=0.05, nsub=5, Ti=0.005, Te=0.005, amp=0.02,
               seed=4000, steps=2000, shape="qs") -> Workload:
    """Quasi-1D cold plasma along B0 = x^ with one linearly polarised
    transverse perturbation dB_y = amp sin(k x), k = 2 pi / Lx, which splits
    into the right-hand (whistler) and left-hand (ion-cyclotron) branches."""
    p = base_params(nx, 1, 1, dx, 1.0, 1.0, dt, nsub, Te=Te, shape=shape, n_floor=0.05,
                    sort_every=0)
    rng = _rng(seed)
    Lx = nx * dx
    k = 2.0 * np.pi / Lx
    x, _, _ = cell_centres(p)
    Az = np.broadcast_to((amp * np.cos(k * x) / k)[None, None, :], (1, 1, nx)).copy()
    B = _curl_of_vector_potential(p, Az=Az)
    B[0] += 1.0
    cell, off = load_cells(p, np.full(nx, ppc), rng, (nx, 1, 1))
    n = cell.shape[0]
    v = math.sqrt(Ti) * _box_muller(rng, (3, n))
    w = np.full(n, dx / ppc)
    return Workload("whistler1d", p, B.astype(np.float32), [_finish(cell, off, v, w)], steps,
                    notes=f"{nx} cells, {ppc} ppc, k={k:.4f}")


def explosion2d(nx=512, nz=512, length=1000.0, ppc=200, n_debris=1 << 20, mach=15.0,
                r_m=150.0, sigma=None, beta=0.1, seed=6000, steps=3000, shape="ngp",
                smooth_passes=0, dt=0.01, nsub=1, eta=0.0, eta_h=0.01, n_floor=0.05,
                sort_every=20) -> Workload:
    """Expanding debris cloud in a magnetised background (the astrophysical
    explosion of Sec. 3.2), x-z plane, periodic.

    Background: n0 = 1, B0 = x^ (in the plane), beta_i = beta_e = beta, so
    T_i = T_e = beta / 2, isothermal electrons, `ppc` ions per cell.  Debris:
    `n_debris` ions of the same charge and mass in a Gaussian cloud of width
    `sigma` (default r_m / 10) at the box centre, each moving radially in the
    plane at `mach` v_A plus the background's thermal spread.  The debris
    holds as many ions as a disc of radius r_m of the background (the
    equal-mass radius; in the x-z plane a disc per unit length in y).
    `smooth_passes` binomial passes are applied both to the moments and to
    the gathered fields (the self-consistent smoothing)."""
    dx = length / nx
    p = base_params(nx, 1, nz, dx, 1.0, dx, dt, nsub, Te=0.5 * beta, eta=eta, eta_h=eta_h,
                    n_floor=n_floor, shape=shape, smooth_passes=smooth_passes,
                    sort_every=sort_every, field_smooth_passes=smooth_passes)
    rng = _rng(seed)
    ncell = nx * nz
    Ti = 0.5 * beta
    B = np.zeros((3, nz, 1, nx))
    B[0] = 1.0
    cell, off = load_cells(p, np.full(ncell, ppc), rng, (nx, 1, nz))
    nb = cell.shape[0]
    v = math.sqrt(Ti) * _box_muller(rng, (3, nb))
    w = np.full(nb, dx * dx / ppc)
    # debris: Gaussian positions about the centre, radial velocities
    sig = 0.1 * r_m if sigma is None else sigma
    Lx, Lz = nx * dx, nz * dx
    rx = sig * _box_muller(rng, n_debris)
    rz = sig * _box_muller(rng, n_debris)
    x = np.mod(0.5 * Lx + rx, Lx)
    z = np.mod(0.5 * Lz + rz, Lz)
    r = np.maximum(np.hypot(rx, rz), 1e-12)
    vd = math.sqrt(Ti) * _box_muller(rng, (3, n_debris))
    vd[0] += mach * rx / r
    vd[2] += mach * rz / r
    fx, fz = x / dx, z / dx
    i = np.minimum(np.floor(fx).astype(np.int64), nx - 1)
    k = np.minimum(np.floor(fz).astype(np.int64), nz - 1)
    offd = np.zeros((3, n_debris))
    offd[0] = np.clip(2.0 * (fx - i) - 1.0, -1.0, 1.0)
    offd[2] = np.clip(2.0 * (fz - k) - 1.0, -1.0, 1.0)
    celld = i + nx * k
    wd = np.full(n_debris, math.pi * r_m * r_m / n_debris)
    cell = np.concatenate([cell, celld])
    order = np.argsort(cell, kind="stable")
    sp = _finish(cell[order], np.concatenate([off, offd], axis=1)[:, order],
                 np.concatenate([v, vd], axis=1)[:, order], np.concatenate([w, wd])[order])
    return Workload("explosion2d", p, B.astype(np.float32), [sp], steps,
                    notes=f"{nx}x{nz} cells, dx={dx:.4f}, {ppc} ppc + {n_debris} debris ions, "
                          f"M_A={mach}, R_m={r_m}, sigma={sig}, {shape}, "
                          f"{smooth_passes} smoothing passes")


def ebeam2d(nx=640, nz=320, lx=80.0, lz=20.0, ppc=64, gamma_d=2.96, u_th=0.3, lam=1.0,
            eta=0.01, dt=0.04, nsub=4, seed=8000, steps=2000, shape="qs",
            sort_every=20) -> Workload:
    """Relativistic electron beam in a resistive background (App. A), x-z
    plane, periodic: electrons (q = -1, m = 1, c = 1 in electron units)
    drifting along x with Lorentz factor gamma_d and a thermal spread u_th
    in u = gamma v, density n0 sech^2((z - Lz/2)/lam) on a floor of 1e-3;
    B_y(z) from the beam current so that curl B = J_beam initially; Ohm's
    law E = eta (curl B - J_beam)."""
    dx, dz = lx / nx, lz / nz
    p = base_params(nx, 1, nz, dx, 1.0, dz, dt, nsub, Te=0.0, eta=eta, n_floor=1e-3,
                    shape=shape, sort_every=sort_every, ohm_model=2, relativistic=1,
                    c_light=1.0)
    rng = _rng(seed)
    _, _, zc = cell_centres(p)
    prof = 1.0 / np.cosh((zc - 0.5 * lz) / lam) ** 2 + 1e-3
    cell, off = load_cells(p, np.full(nx * nz, ppc), rng, (nx, 1, nz))
    n = cell.shape[0]
    k = cell // nx
    u = u_th * _box_muller(rng, (3, n))
    ud = math.sqrt(gamma_d * gamma_d - 1.0)
    u[0] += ud
    w = prof[k] * dx * dz / ppc
    # B_y with -dB_y/dz = J_x = q n v_d (v_d = ud / gamma_d), zero mean
    jx = -1.0 * prof * ud / gamma_d
    By = -np.cumsum(jx) * dz
    By -= By.mean()
    B = np.zeros((3, nz, 1, nx))
    B[1] = By[:, None, None]
    return Workload("ebeam2d", p, B.astype(np.float32), [_finish(cell, off, u, w, q=-1.0, m=1.0)],
                    steps, notes=f"{nx}x{nz} cells, {ppc} ppc, gamma_d={gamma_d}, eta={eta}")


WORKLOADS = {
    "alfven2d": alfven2d,
    "harris2d": harris2d,
    "beam3d": beam3d,
    "harris3d": harris3d,
    "whistler1d": whistler1d,
    "explosion2d": explosion2d,
    "ebeam2d": ebeam2d,
}


def harris_device(nx=512, ny=256, nz=256, ppc=32, dx=0.5, seed=3000, steps=1000, shape="qs",
                  guide=0.1, sort_every=20, lam=1.0, nb=0.2, pert=0.1, dt=0.02, nsub=10,
                  device="cuda", chunk=1 << 26) -> Workload:
    """The Harris sheet of ``harris`` generated on the GPU with torch, for
    sizes whose host generation would need more memory and time than the
    run (the 3D sheet at 512x256x256 with 32 ppc is 1.07e9 ions, 34 GB of
    FP32 particle data).  Same recipe: ions in cell order, every cell holds
    ``ppc`` ions split between the two sheets and the background by the
    local densities (sheet ions first), uniform relative coordinates,
    drifting Maxwellian velocities and per-population weights; the random
    numbers come from torch's seeded CUDA generator, so the arrays are not
    bit-identical to ``harris`` with the same seed.  The B0 field is built on
    the host exactly as in ``harris``.  Species arrays are CUDA tensors."""
    import torch
    p = base_params(nx, ny, nz, dx, dx, dx, dt, nsub, Te=1.0 / 12.0, eta=1e-3, eta_h=1e-4,
                    n_floor=0.05, shape=shape, sort_every=sort_every)
    Ti = 5.0 / 12.0
    Lx, Lz = nx * dx, nz * dx
    x, y, z = cell_centres(p)
    Bx_z, ns1_z, ns2_z, _ = harris_profile(z, Lz, lam, nb)
    wdt = 2.0 * lam
    A0 = pert * wdt * math.exp(0.5)
    X, Z = np.meshgrid(x, z)
    Ay2 = A0 * np.exp(-((X - 0.5 * Lx) ** 2 + (Z - 0.75 * Lz) ** 2) / (2.0 * wdt ** 2))
    Ay = np.broadcast_to(Ay2[:, None, :], (nz, ny, nx)).copy()
    B = _curl_of_vector_potential(p, Ay=Ay)
    B[0] += Bx_z[:, None, None]
    B[1] += guide
    n_tot = ns1_z + ns2_z + nb
    c1 = np.floor(ppc * ns1_z / n_tot + 0.5).astype(np.int64)
    c2 = np.floor(ppc * ns2_z / n_tot + 0.5).astype(np.int64)
    cb = ppc - c1 - c2
    vc = dx * p["dy"] * dx
    w1 = ns1_z * vc / np.maximum(c1, 1)
    w2 = ns2_z * vc / np.maximum(c2, 1)
    wb = nb * vc / np.maximum(cb, 1)
    dev = torch.device(device)
    tc1 = torch.as_tensor(c1, device=dev)
    tc2 = torch.as_tensor(c2, device=dev)
    tw = torch.as_tensor(np.stack([w1, w2, wb]), dtype=torch.float32, device=dev)  # [3][nz]
    ncell = nx * ny * nz
    n = ncell * ppc
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty((3, n), dtype=torch.float32, device=dev)
    v = torch.empty((3, n), dtype=torch.float32, device=dev)
    w = torch.empty(n, dtype=torch.float32, device=dev)
    U = 2.0 * Ti / lam
    below1 = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        idx = torch.arange(a, b, device=dev, dtype=torch.int64)
        c = idx // ppc
        j = idx - c * ppc
        k = c // (nx * ny)
        pop = torch.where(j < tc1[k], 0, torch.where(j < tc1[k] + tc2[k], 1, 2))
        cell[a:b] = c.to(torch.int32)
        o = torch.rand((3, b - a), generator=gen, device=dev, dtype=torch.float32) * 2.0 - 1.0
        off[:, a:b] = o.clamp_(max=below1)
        vv = torch.randn((3, b - a), generator=gen, device=dev, dtype=torch.float32) * math.sqrt(Ti)
        vv[1] += torch.where(pop == 0, U, torch.where(pop == 1, -U, 0.0)).to(torch.float32)
        v[:, a:b] = vv
        w[a:b] = tw[pop, k]
    sp = SpeciesInput(1.0, 1.0, cell, off, v, w)
    return Workload("harris3d", p, B.astype(np.float32), [sp], steps,
                    notes=f"{nx}x{ny}x{nz} cells, {ppc} ppc, dx={dx}, guide={guide}, seed={seed}, "
                          f"generated on the GPU")


def drifting_slab(nx=32, ny=1, nz=16, ppc=32, dx=0.5, U=0.4, Ti=0.04, Te=0.02, Bz=0.3,
                  seed=90, dt=0.02, nsub=4, shape="qs", open_faces=1, sort_every=0,
                  w_scale=1.0) -> Workload:
    """A uniform plasma flowing at U along x through a box (open faces on the
    axes in ``open_faces``, bits x = 1, y = 2, z = 4) in the field
    B = (1, 0, Bz), with ion temperature Ti: the workload of the open-face
    tests.  Weights are n V_c / ppc times w_scale."""
    dy = dx if ny > 1 else 1.0
    p = base_params(nx, ny, nz, dx, dy, dx, dt, nsub, Te=Te, shape=shape, sort_every=sort_every,
                    eta=1e-3, eta_h=1e-4)
    p["open_faces"] = open_faces
    rng = _rng(seed)
    B = np.zeros((3, nz, ny, nx))
    B[0] = 1.0
    B[2] = Bz
    ncell = nx * ny * nz
    cell, off = load_cells(p, np.full(ncell, ppc), rng, (nx, ny, nz))
    n = cell.shape[0]
    v = np.sqrt(Ti) * _box_muller(rng, (3, n))
    v[0] += U
    w = np.full(n, dx * dy * dx / ppc * w_scale)
    wl = Workload("drifting_slab", p, B.astype(np.float32), [_finish(cell, off, v, w)], 1,
                  notes=f"{nx}x{ny}x{nz} cells, {ppc} ppc, U={U}, open_faces={open_faces}")
    # the same drifting Maxwellian enters through every open face
    w_inj = float(np.float32(dx * dy * dx / ppc * w_scale))
    for a in range(3):
        if (open_faces >> a) & 1:
            u = [U, 0.0, 0.0]
            wl.inject += [(0, 2 * a, 1.0, u, Ti, w_inj), (0, 2 * a + 1, 1.0, u, Ti, w_inj)]
    wl.reserve = 1.25 if open_faces else 0.0
    return wl
