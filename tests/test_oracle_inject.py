"""Pins of the oracle's injection through open faces (Sec. 2.3; reading R24):
the Philox4x32-10 generator against its published known-answer vectors, the
one-sided flux of a drifting Maxwellian against closed forms, the
flux-weighted speed sampling against the Rayleigh inverse (no drift) and a
quadrature of the distribution (drift), and a steady flow through an open
box: injection balances outflow."""
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert O.philox4x32_10(ctr, key).tolist() == want


def grid(nx, nz, open_axes=(1, 0, 0), dt=0.05):
    return O.make_grid(nx, 1, nz, 0.5, 1.0, 0.5, dt, 2, 0.0, 1.0, 0.0, 0.0, 0.01, "qs",
                       open_axes=open_axes)


def test_expected_count_is_the_one_sided_flux():
    g = grid(8, 4)
    # no drift: Gamma = n vt / sqrt(2 pi); face cell area dy dz = 0.5
    f = O.inject_face(0, 2.0, (0.0, 0.0, 0.0), 0.5, 0.01)
    N = 2.0 * np.sqrt(0.5) / np.sqrt(2 * np.pi) * 0.5 * 0.05 / 0.01
    assert O.inject_nfix(g, 1.0, f) == int(np.floor(N * 2 ** 24 + 0.5))
    # a cold beam into the +x face (inward = -x) at speed 3: Gamma = n * 3
    f = O.inject_face(1, 1.0, (-3.0, 0.0, 0.0), 0.0, 0.02)
    assert O.inject_nfix(g, 1.0, f) == int(np.floor(3.0 * 0.5 * 0.05 / 0.02 * 2 ** 24 + 0.5))
    # flowing out: no flux from a cold beam
    f = O.inject_face(0, 1.0, (-3.0, 0.0, 0.0), 0.0, 0.02)
    assert O.inject_nfix(g, 1.0, f) == 0


def test_undrifted_inward_speeds_follow_the_rayleigh_inverse():
    """With no drift the flux-weighted speed density is t exp(-t^2/2): the
    injected normal speed is vt sqrt(-2 ln(1 - u0)) for the cell's u0."""
    g = grid(8, 4, dt=0.5)
    f = O.inject_face(0, 50.0, (0.0, 0.0, 0.0), 0.25, 0.01)
    cell, off, v = O.inject(g, 0, 1.0, f, seed=11, step=3)
    assert cell.shape[0] > 50
    # reconstruct u0 of each ion from the generator and compare
    key = [11, 0]
    k_of_cell = {}
    for idx in range(cell.shape[0]):
        c = int(cell[idx] // 8)  # tangential (z) cell index of the x face
        k = k_of_cell.get(c, 0)
        k_of_cell[c] = k + 1
        r = O.philox4x32_10([3, c, k, 0 << 8 | 0 << 4], key)
        u0 = (int(r[0]) >> 8) / 2 ** 24
        assert abs(v[0, idx] - 0.5 * np.sqrt(-2 * np.log(1 - u0))) < 1e-9


def test_drifting_inward_speeds_invert_the_flux_distribution():
    quad = pytest.importorskip("scipy.integrate").quad
    g = grid(4, 2, dt=0.5)
    a = 1.3  # U / vt
    f = O.inject_face(0, 200.0, (a * 0.5, 0.0, 0.0), 0.25, 0.01)
    cell, off, v = O.inject(g, 0, 1.0, f, seed=5, step=0)
    dens = lambda t: t * np.exp(-0.5 * (t - a) ** 2)  # noqa: E731
    norm = quad(dens, 0, np.inf)[0]
    key = [5, 0]
    seen = {}
    for idx in range(min(40, cell.shape[0])):
        c = int(cell[idx] // 4)
        k = seen.get(c, 0)
        seen[c] = k + 1
        r = O.philox4x32_10([0, c, k, 0], key)
        u0 = (int(r[0]) >> 8) / 2 ** 24
        t = v[0, idx] / 0.5
        assert abs(quad(dens, 0, t)[0] / norm - u0) < 1e-9


def test_steady_flow_through_an_open_box():
    """A uniform plasma flowing along B = x through a box open in x, with the
    same drifting Maxwellian injected at both faces: inflow balances outflow,
    so the ion count and the density profile stay level (no field: T_e = 0
    and u parallel to B)."""
    nx, nz, ppc, U, T = 16, 4, 64, 0.4, 0.04
    dt = 0.05
    g = O.make_grid(nx, 1, nz, 0.5, 1.0, 0.5, dt, 2, 0.0, 1.0, 0.0, 0.0, 0.01, "ngp",
                    open_axes=(1, 0, 0))
    rng = np.random.default_rng(1)
    n = nx * nz * ppc
    cell = np.repeat(np.arange(nx * nz), ppc)
    off = np.zeros((3, n))
    off[0] = rng.uniform(-1, 1, n)
    off[2] = rng.uniform(-1, 1, n)
    v = rng.normal(0, np.sqrt(T), (3, n))
    v[0] += U
    w = np.full(n, 0.25 / ppc)
    B = np.zeros((3, nx * nz))
    B[0] = 1.0
    faces = [(0, O.inject_face(0, 1.0, (U, 0, 0), T, 0.25 / ppc)),
             (0, O.inject_face(1, 1.0, (U, 0, 0), T, 0.25 / ppc))]
    sim = O.Sim(g, [O.Species(1.0, 1.0, cell, off, v, w)], B, inject=faces, seed=7)
    counts = []
    for _ in range(60):
        sim.step(1)
        counts.append(sim.species[0].n)
    counts = np.array(counts)
    assert abs(counts[-20:].mean() / n - 1.0) < 0.03, counts[-20:].mean() / n
    prof = sim.n_prev.reshape(nz, nx).mean(axis=0)
    assert np.abs(prof / prof.mean() - 1.0).max() < 0.15
