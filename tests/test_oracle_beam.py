"""Pins of the oracle's kinetic-electron beam pieces (App. A): the
relativistic Boris push (reading R19) and the resistive-background Ohm's law
E = eta (curl B - J_k) (reading R18).  Closed forms: a relativistic Boris
rotation turns u by 2 atan(h |B| / gamma) at constant |u|; an electric kick
adds q E dt / m to u; with no fields a particle moves by u / gamma dt; the
centred curl of a mode B_y(z) = b sin(k z) is J_x = -b cos(k z) sin(k dz)/dz,
and the resistive step multiplies that mode by 1 + mu h + (mu h)^2 / 2 with
mu = -eta sin^2(k dz)/dz^2.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(77)


@pytest.mark.parametrize("gamma", [1.0001, 2.0, 10.0])
def test_relativistic_rotation_angle_and_speed(gamma):
    c = 1.0
    umag = c * math.sqrt(gamma ** 2 - 1)
    B = np.array([0.0, 0.0, 1.7])
    qmdt = 0.3
    u0 = np.array([umag, 0.0, 0.0])
    u1 = O.boris_rel(qmdt, c, [0, 0, 0], B, u0)
    assert abs(np.linalg.norm(u1) - umag) < 1e-12 * umag
    ang = math.atan2(u0[0] * u1[1] - u0[1] * u1[0], u0 @ u1)
    # q > 0 gyrates clockwise about +z: the angle is negative
    assert abs(ang + 2 * math.atan(0.5 * qmdt * 1.7 / gamma)) < 1e-12


def test_electric_kicks_add_momentum_and_speed_stays_below_c():
    c = 1.0
    E = np.array([0.0, 4.0, 0.0])
    u = np.zeros(3)
    for n in range(1, 51):
        u = O.boris_rel(0.5, c, E, [0, 0, 0], u)
        assert abs(u[1] - n * 0.5 * 4.0) < 1e-12 * n
        assert np.linalg.norm(u) / math.sqrt(1 + u @ u / c ** 2) < c


def test_nonrelativistic_limit():
    for _ in range(10):
        E, B, v = RNG.normal(size=3), RNG.normal(size=3), RNG.normal(size=3) * 0.1
        a = O.boris(0.2, E, B, v)
        b = O.boris_rel(0.2, 1e8, E, B, v)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def beam_grid(eta=0.0, nsub=2, relativistic=1, c=1.0, shape="qs"):
    return O.make_grid(16, 1, 8, 0.25, 1.0, 0.25, 0.05, nsub=nsub, Te=0.0, gamma_e=1.0, eta=eta,
                       eta_h=0.0, n_floor=0.05, shape=shape, ohm_model=2,
                       relativistic=relativistic, c_light=c)


def test_free_streaming_moves_by_u_over_gamma_and_reports_gamma_minus_one():
    g = beam_grid()
    u = np.array([[2.0], [0.5], [0.0]])
    gam = math.sqrt(1 + (u ** 2).sum())
    sp = O.Species(-1.0, 1.0, np.array([3 + 16 * 4]), np.array([[0.1], [0.0], [-0.2]]), u,
                   np.array([0.5]))
    sim = O.Sim(g, [sp], np.zeros((3, 128)))
    x0 = (3 + 0.5 + 0.5 * 0.1) * g.dx
    for n in range(1, 4):
        d = sim.step(1)
        s = sim.species[0]
        x = (s.cell[0] % 16 + 0.5 + 0.5 * s.off[0, 0]) * g.dx
        dxp = (x - x0 - n * g.dt * u[0, 0] / gam) % (16 * g.dx)
        assert min(dxp, 16 * g.dx - dxp) < 1e-12
        assert np.array_equal(s.v[:, 0], u[:, 0])
        assert abs(d["W_K"] - 0.5 * (gam - 1.0)) < 1e-13
        assert np.allclose(d["P"], 0.5 * u[:, 0], atol=1e-15)
    # the deposited current is q w v / V_c summed over the cells, v = u / gamma
    n_, J = O.deposit(g, sim.species)
    vc = g.dx * g.dy * g.dz
    assert np.allclose(J.sum(axis=1) * vc, -0.5 * u[:, 0] / gam, rtol=1e-13, atol=1e-15)


def test_resistive_ohm_is_eta_times_background_current():
    g = beam_grid(eta=0.3)
    nc = 128
    _, z = (np.arange(nc) % 16 + 0.5) * g.dx, (np.arange(nc) // 16 + 0.5) * g.dz
    k = 2 * math.pi / (8 * g.dz)
    b = 0.4
    B = np.zeros((3, nc))
    B[1] = b * np.sin(k * z)
    B[2] = 2.0  # a uniform component carries no current
    Jk = np.zeros((3, nc))
    Jk[0] = 0.05
    Jk[2] = -0.02
    E = O.ohm(g, B, np.ones(nc), Jk)
    jx = -b * np.cos(k * z) * math.sin(k * g.dz) / g.dz
    assert np.abs(E[0] - 0.3 * (jx - 0.05)).max() < 1e-14
    assert np.abs(E[1]).max() < 1e-15
    assert np.abs(E[2] - 0.3 * 0.02).max() < 1e-15


def test_resistive_diffusion_of_a_mode_matches_rk2_amplification():
    g = beam_grid(eta=0.02, nsub=5)
    nc = 128
    z = (np.arange(nc) // 16 + 0.5) * g.dz
    k = 2 * math.pi / (8 * g.dz)
    B = np.zeros((3, nc))
    B[1] = 0.4 * np.sin(k * z)
    Jk = np.zeros((3, nc))
    Jk[0] = 0.1  # uniform: no curl
    h = g.dt / g.nsub
    mu = -0.02 * math.sin(k * g.dz) ** 2 / g.dz ** 2
    G = (1 + mu * h + (mu * h) ** 2 / 2) ** g.nsub
    B1 = O.field_advance(g, B, np.ones(nc), Jk)
    assert np.abs(B1[1] - G * B[1]).max() < 1e-14
    assert np.abs(B1[[0, 2]]).max() < 1e-15
