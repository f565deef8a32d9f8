"""Pins of the oracle's B = B0 + B1 split (Sec. 2.3; reading R20): a fixed
external field B0, only B1 advanced, the current J = curl B1, and the total
field in every cross product and in the push.  Each pin fails for a plausible
mistake: J taken from the total field, B0 dropped from the Hall / ion term,
B0 dropped from the push, B0 advanced, W_B of B1 only."""
import numpy as np

import oracle as O


def grid(nx, nz, B0ext=None, **kw):
    p = dict(dx=0.5, dy=1.0, dz=0.5, dt=0.01, nsub=4, Te=0.0, n_floor=0.01, shape="qs")
    p.update(kw)
    return O.make_grid(nx, 1, nz, p["dx"], p["dy"], p["dz"], p["dt"], p["nsub"], p["Te"], 1.0,
                       0.0, 0.0, p["n_floor"], p["shape"], B0ext=B0ext)


def cold_lattice(nx, nz, v=(0.0, 0.0, 0.0), per_cell=1):
    """per_cell ions at every cell centre, equal weights (uniform n = 1)."""
    cell = np.repeat(np.arange(nx * nz), per_cell)
    n = cell.shape[0]
    off = np.zeros((3, n))
    vv = np.tile(np.asarray(v, float)[:, None], (1, n))
    w = np.full(n, 0.5 * 0.5 / per_cell)
    return O.Species(1.0, 1.0, cell, off, vv, w)


def curly_b0(nx, nz, dx=0.5):
    """An external field whose centred discrete curl is not zero."""
    x = (np.arange(nx) + 0.5) * dx
    b = np.zeros((3, 1, nz, nx))
    b[0] = 1.0
    b[2] = 0.2 * np.sin(2 * np.pi * x / (nx * dx))[None, None, :]
    return b.reshape(3, -1)


def test_plasma_at_rest_in_external_field_is_stationary():
    nx, nz = 16, 8
    b0 = curly_b0(nx, nz)
    sim = O.Sim(grid(nx, nz, B0ext=b0), [cold_lattice(nx, nz)], b0)
    sim.step(5)
    assert np.array_equal(sim.B, np.zeros_like(sim.B))  # B1 untouched
    assert np.abs(sim.E).max() == 0.0
    assert np.array_equal(sim.B_total(), b0)
    # without the split the same total field carries J = curl B0 and evolves
    ref = O.Sim(grid(nx, nz), [cold_lattice(nx, nz)], b0)
    ref.step(5)
    assert np.abs(ref.B - b0).max() > 1e-6


def test_drifting_plasma_is_an_exact_exb_equilibrium():
    """Uniform drift u across an external B0 = z: Ohm's law gives the
    motional field E = -u x B, the ions drift at exactly u, B1 stays 0.  A
    push or Ohm's law without B0 breaks it."""
    nx, nz = 12, 8
    b0 = np.zeros((3, nx * nz))
    b0[2] = 1.0
    u = (0.3, 0.0, 0.0)
    sim = O.Sim(grid(nx, nz, B0ext=b0), [cold_lattice(nx, nz, v=u, per_cell=2)], b0)
    sim.step(10)
    v = sim.species[0].v
    assert np.abs(v[0] - 0.3).max() < 1e-12 and np.abs(v[1:]).max() < 1e-12
    assert np.abs(sim.B).max() < 1e-12
    assert np.allclose(sim.E[1], 0.3, atol=1e-12)  # E_y = -(u x B)_y = u_x B_z


def test_uniform_external_field_matches_unsplit_run():
    rng = np.random.default_rng(3)
    nx, nz = 12, 10
    n = 8 * nx * nz
    cell = rng.integers(0, nx * nz, n)
    off = np.zeros((3, n))
    off[0] = rng.uniform(-1, 1, n)
    off[2] = rng.uniform(-1, 1, n)
    v = rng.normal(0, 0.3, (3, n))
    w = np.full(n, 0.25 / 8)
    Bt = np.zeros((3, nx * nz))
    Bt[0] = 1.0 + 0.05 * rng.normal(size=nx * nz)
    Bt[2] = 0.3
    b0 = np.zeros_like(Bt)
    b0[0] = 1.0
    b0[2] = 0.3
    kw = dict(Te=0.1, eta=1e-3, eta_h=1e-4)
    a = O.Sim(grid(nx, nz, **kw), [O.Species(1.0, 1.0, cell, off, v, w)], Bt)
    b = O.Sim(grid(nx, nz, B0ext=b0, **kw), [O.Species(1.0, 1.0, cell, off, v, w)], Bt)
    a.step(3)
    b.step(3)
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)  # noqa: E731
    assert rel(b.B_total(), a.B) < 1e-12
    assert rel(b.E, a.E) < 1e-12
    assert rel(b.species[0].v, a.species[0].v) < 1e-12
    assert abs(b.diags[-1]["W_B"] - a.diags[-1]["W_B"]) < 1e-12 * a.diags[-1]["W_B"]


def test_hall_term_uses_curl_of_b1_and_total_field():
    """B1 = d sin(kx) y, B0 = x (external), n = 1, J_i = 0, no pressure or
    resistivity: E = J x (B0 + B1) with J = z d k_eff cos(kx),
    k_eff = sin(k dx) / dx (centred difference, Eq. 12)."""
    nx, nz, dx = 32, 4, 0.5
    g = grid(nx, nz, B0ext=np.vstack([np.ones(nx * nz), np.zeros(nx * nz), np.zeros(nx * nz)]))
    x = np.tile((np.arange(nx) + 0.5) * dx, nz)
    k, d = 2 * np.pi / (nx * dx), 0.01
    B1 = np.zeros((3, nx * nz))
    B1[1] = d * np.sin(k * x)
    E = O.ohm(g, B1, np.ones(nx * nz), np.zeros((3, nx * nz)))
    Jz = d * np.sin(k * dx) / dx * np.cos(k * x)
    assert np.allclose(E[0], -Jz * B1[1], atol=1e-15)
    assert np.allclose(E[1], Jz * 1.0, atol=1e-15)
    assert np.abs(E[2]).max() < 1e-15


def test_diagnostics_take_total_field_energy_and_b1_divergence():
    nx, nz = 16, 8
    b0 = curly_b0(nx, nz)
    sim = O.Sim(grid(nx, nz, B0ext=b0), [cold_lattice(nx, nz)], b0)
    d = sim.step(1)
    vc = 0.5 * 1.0 * 0.5
    assert abs(d["W_B"] - 0.5 * np.sum(b0 ** 2) * vc) < 1e-12 * d["W_B"]
    assert d["max_divB"] == 0.0  # max |div B1|, and B1 = 0
