"""Pins of the oracle's self-consistent field smoothing (Sec. 2.2: one or more
passes of a field and moment smoother).  The ions gather from S^p E and
S^p B, where S is the binomial (1/4, 1/2, 1/4) operator the moments are
smoothed with; the field state itself is not smoothed.

Closed forms used:
  * a Fourier mode sin(k x_c) on the cell centres is an eigenvector of one
    binomial pass along x with eigenvalue 1/2 + 1/2 cos(k dx) = cos^2(k dx/2),
    and of a pass along an axis it does not vary on with eigenvalue 1;
  * with B = 0 the Boris step changes v by (q/m) dt E_gathered (Eq. 9), so
    the kick from a smoothed mode is cos^{2p}(k dx/2) times the kick from
    the unsmoothed mode, ion by ion;
  * with E = 0 the Boris step rotates v about B by 2 atan(|t|), t =
    (q dt / 2m) B_gathered, so tan(half the rotation) scales the same way;
  * S is symmetric, so gathering from S^p F equals pairing F with S^p of the
    ion's deposit weights (the transpose; no self-force).
CPU only."""
import math

import numpy as np
import pytest

import oracle as O


def mode_grid(p, shape="qs", nx=32, nz=8, dx=0.5, dt=0.05):
    return O.make_grid(nx, 1, nz, dx, 1.0, dx, dt, nsub=1, Te=0.0, gamma_e=1.0, eta=0.0,
                       eta_h=0.0, n_floor=0.05, shape=shape, field_smooth_passes=p)


def random_ions(g, n, seed, w=1.0):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, g.nx * g.ny * g.nz, n)
    off = rng.uniform(-1.0, 1.0, (3, n))
    off[1] = 0.0
    v = rng.normal(0.0, 0.3, (3, n))
    return O.Species(1.0, 1.0, cell, off, v, np.full(n, w))


def one_step(g, sp, E, B):
    sim = O.Sim(g, [sp], B)
    sim.E = np.ascontiguousarray(E, dtype=np.float64).copy()
    sim.B = np.ascontiguousarray(B, dtype=np.float64).copy()
    sim.step(1)
    return sim


def x_mode(g, m=1):
    i = np.arange(g.nx * g.ny * g.nz) % g.nx
    xc = (i + 0.5) * g.dx
    return np.sin(2.0 * math.pi * m * xc / (g.nx * g.dx))


@pytest.mark.parametrize("shape", ["ngp", "qs", "cic"])
@pytest.mark.parametrize("p", [1, 3])
def test_smoothed_E_kick_is_eigenvalue_times_kick(shape, p):
    g0, gp = mode_grid(0, shape), mode_grid(p, shape)
    sp = random_ions(g0, 400, seed=7)
    E = np.zeros((3, g0.nx * g0.nz))
    E[1] = 0.8 * x_mode(g0)
    B = np.zeros_like(E)
    s0 = one_step(g0, sp.copy(), E, B)
    sp_ = one_step(gp, sp.copy(), E, B)
    dv0 = s0.species[0].v[1] - sp.v[1]
    dvp = sp_.species[0].v[1] - sp.v[1]
    lam = math.cos(math.pi / g0.nx) ** (2 * p)
    assert np.allclose(dvp, lam * dv0, rtol=1e-11, atol=1e-14)
    # x and z velocities see no E component
    assert np.allclose(sp_.species[0].v[0], sp.v[0], rtol=0, atol=1e-15)
    assert np.allclose(sp_.species[0].v[2], sp.v[2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2])
def test_smoothed_B_rotation_is_eigenvalue_scaled(p):
    g0, gp = mode_grid(0), mode_grid(p)
    sp = random_ions(g0, 300, seed=8)
    B = np.zeros((3, g0.nx * g0.nz))
    B[2] = 3.0 * x_mode(g0, m=2)
    E = np.zeros_like(B)

    def half_tan(sim):
        v0 = sp.v[:2]
        v1 = sim.species[0].v[:2]
        ang = np.arctan2(v0[0] * v1[1] - v0[1] * v1[0], (v0 * v1).sum(0))
        return np.tan(0.5 * ang)

    t0 = half_tan(one_step(g0, sp.copy(), E, B))
    tp = half_tan(one_step(gp, sp.copy(), E, B))
    lam = math.cos(2.0 * math.pi / g0.nx) ** (2 * p)
    assert np.allclose(tp, lam * t0, rtol=1e-10, atol=1e-14)


def test_field_state_is_not_smoothed():
    """Ions of zero weight deposit nothing, so B^{n+1} and E^{n+1} must not
    depend on the field smoothing of the gathered copies."""
    rng = np.random.default_rng(3)
    g0 = O.make_grid(12, 1, 10, 0.5, 1.0, 0.5, 0.02, nsub=2, Te=0.1, eta=1e-3, eta_h=1e-4,
                     n_floor=0.05, shape="qs")
    gp = O.make_grid(12, 1, 10, 0.5, 1.0, 0.5, 0.02, nsub=2, Te=0.1, eta=1e-3, eta_h=1e-4,
                     n_floor=0.05, shape="qs", field_smooth_passes=4)
    sp = random_ions(g0, 50, seed=4, w=0.0)
    B = rng.normal(size=(3, 120))
    E = rng.normal(size=(3, 120))
    s0 = one_step(g0, sp.copy(), E, B)
    s1 = one_step(gp, sp.copy(), E, B)
    assert np.array_equal(s0.B, s1.B)
    assert np.array_equal(s0.E, s1.E)
    # while the ions themselves do see the smoothed field
    assert not np.allclose(s0.species[0].v, s1.species[0].v)


@pytest.mark.parametrize("shape", ["ngp", "qs", "cic"])
@pytest.mark.parametrize("dims", [(9, 1, 7), (6, 5, 7)])
def test_smoothed_gather_is_transpose_of_smoothed_deposit(shape, dims):
    nx, ny, nz = dims
    rng = np.random.default_rng(11)
    g = O.make_grid(nx, ny, nz, 0.5, 0.5 if ny > 1 else 1.0, 0.5, 0.01, shape=shape)
    vc = g.dx * g.dy * g.dz
    F = rng.normal(size=(3, nx * ny * nz))
    for p in (1, 2):
        SF = O.smooth(g, F, p).reshape(3, -1)
        for _ in range(5):
            cell = int(rng.integers(0, nx * ny * nz))
            d = rng.uniform(-1, 1, 3)
            if ny == 1:
                d[1] = 0.0
            ion = O.Species(1.0, 1.0, np.array([cell]), d.reshape(3, 1), np.zeros((3, 1)),
                            np.array([vc]))
            W, _ = O.deposit(g, [ion])  # the ion's deposit weights W_c
            SW = O.smooth(g, W, p)
            lhs = O.gather(g, SF, cell, d)
            rhs = (F * SW[None, :]).sum(axis=1)
            assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-13), (lhs, rhs)
