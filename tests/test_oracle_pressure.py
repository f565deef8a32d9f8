"""Pins of the oracle's electron energy equation (Sec. 2.1, Eq. dpdt; reading
R16):  dp_e/dt = -gamma div(p_e u_e) + (gamma - 1) u_e . grad p_e
+ (gamma - 1) kappa lap(T_e),  u_e = -(curl B - J_i)/n_f,  T_e = p_e / n_f,
advanced with B in explicit-midpoint subcycles; and of the electrostatic
model (Sec. 4, Eq. esohm; reading R17): E = -grad p_e / n_f, B not advanced.

Closed forms on the cell-centred grid (centred differences, Eq. 12): the
centred derivative of exp(i k x) is i sin(k dx)/dx exp(i k x) and the
3-point second difference is -(4/dx^2) sin^2(k dx/2) exp(i k x).  An
explicit-midpoint step of dp/dt = lambda p multiplies by
1 + lambda h + (lambda h)^2 / 2.  The tests use gamma = 5/3 so that the
two convective terms do not collapse by accident.  CPU only."""
import math

import numpy as np

import oracle as O

GAM = 5.0 / 3.0


def grid2d(nx=24, nz=16, dx=0.5, dt=0.02, nsub=4, kappa=0.0, eta=1e-3, eta_h=1e-4):
    return O.make_grid(nx, 1, nz, dx, 1.0, dx, dt, nsub=nsub, Te=0.1, gamma_e=GAM, eta=eta,
                       eta_h=eta_h, n_floor=0.05, shape="qs", pe_eq=1, kappa=kappa)


def centres(g):
    c = np.arange(g.nx * g.ny * g.nz)
    i = c % g.nx
    k = c // (g.nx * g.ny)
    return (i + 0.5) * g.dx, (k + 0.5) * g.dz


def test_uniform_state_is_steady():
    g = grid2d(kappa=0.05)
    nc = g.nx * g.nz
    B = np.tile(np.array([[0.3], [0.2], [1.0]]), (1, nc))
    n = np.full(nc, 1.3)
    Ji = np.tile(np.array([[0.1], [-0.2], [0.05]]), (1, nc))
    pe = np.full(nc, 0.7)
    assert np.abs(O.dpdt(g, B, pe, n, Ji)).max() < 1e-14
    B1, p1 = O.field_advance_pe(g, B, pe, n, Ji)
    assert np.abs(p1 - pe).max() < 1e-14 and np.abs(B1 - B).max() < 1e-14


def test_advection_by_uniform_ion_flow_matches_rk2_amplification():
    """J = 0, u_e = J_i / n uniform along x: the two convective terms sum to
    -u . grad p, so a mode moves with the centred-difference phase speed."""
    g = grid2d()
    nc = g.nx * g.nz
    x, _ = centres(g)
    k = 2 * math.pi * 2 / (g.nx * g.dx)
    u0, p0, dl = 0.8, 0.5, 0.01
    B = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, nc))
    n = np.ones(nc)
    Ji = np.zeros((3, nc))
    Ji[0] = u0
    pe = p0 + dl * np.sin(k * x)
    h = g.dt / g.nsub
    lam = -1j * u0 * math.sin(k * g.dx) / g.dx
    G = (1 + lam * h + (lam * h) ** 2 / 2) ** g.nsub
    B1, p1 = O.field_advance_pe(g, B, pe, n, Ji)
    expect = p0 + dl * np.imag(G * np.exp(1j * k * x))
    assert np.abs(p1 - expect).max() < 1e-14
    assert np.abs(B1 - B).max() < 1e-14  # E_x varies along x only: curl E = 0


def test_heat_conduction_mode_matches_rk2_amplification():
    """u_e = 0: dp/dt = (gamma - 1) kappa lap(p / n) for uniform n."""
    g = grid2d(kappa=0.3, nsub=3)
    nc = g.nx * g.nz
    _, z = centres(g)
    k = 2 * math.pi / (g.nz * g.dz)
    n0, p0, dl = 1.5, 0.6, 0.02
    B = np.tile(np.array([[1.0], [0.0], [0.0]]), (1, nc))
    n = np.full(nc, n0)
    Ji = np.zeros((3, nc))
    pe = p0 + dl * np.sin(k * z)
    h = g.dt / g.nsub
    mu = -(GAM - 1) * 0.3 / n0 * 4 * math.sin(k * g.dz / 2) ** 2 / g.dz ** 2
    G = (1 + mu * h + (mu * h) ** 2 / 2) ** g.nsub
    B1, p1 = O.field_advance_pe(g, B, pe, n, Ji)
    assert np.abs(p1 - (p0 + dl * G * np.sin(k * z))).max() < 1e-14
    assert np.abs(B1 - B).max() < 1e-13


def test_compression_term_is_gamma_p_div_u():
    """Uniform p_e in a sinusoidal ion flow (J = 0): dp/dt = -gamma p div u_e."""
    g = grid2d()
    nc = g.nx * g.nz
    x, _ = centres(g)
    k = 2 * math.pi / (g.nx * g.dx)
    u0, p0 = 0.4, 0.9
    B = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, nc))
    n = np.ones(nc)
    Ji = np.zeros((3, nc))
    Ji[0] = u0 * np.sin(k * x)
    pe = np.full(nc, p0)
    expect = -GAM * p0 * u0 * np.cos(k * x) * math.sin(k * g.dx) / g.dx
    assert np.abs(O.dpdt(g, B, pe, n, Ji) - expect).max() < 1e-13


def test_electron_flow_comes_from_minus_curl_B():
    """J_i = 0 and B_y(z): J_x = -dB_y/dz, u_e = -J / n carries p_e along x."""
    g = grid2d()
    nc = g.nx * g.nz
    x, z = centres(g)
    kx = 2 * math.pi / (g.nx * g.dx)
    kz = 2 * math.pi / (g.nz * g.dz)
    b, p0, dl = 0.2, 0.5, 0.03
    B = np.zeros((3, nc))
    B[1] = b * np.sin(kz * z)
    B[2] = 1.0
    n = np.ones(nc)
    Ji = np.zeros((3, nc))
    pe = p0 + dl * np.sin(kx * x)
    ux = b * np.cos(kz * z) * math.sin(kz * g.dz) / g.dz
    expect = -ux * dl * np.cos(kx * x) * math.sin(kx * g.dx) / g.dx
    assert np.abs(O.dpdt(g, B, pe, n, Ji) - expect).max() < 1e-13


def test_ohm_uses_the_pressure_field():
    """grad p_e in Ohm's law comes from the field: a pressure mode on an
    otherwise field-free, current-free state gives E = -grad p_e / n."""
    g = grid2d(eta=0.0, eta_h=0.0)
    nc = g.nx * g.nz
    x, _ = centres(g)
    k = 2 * math.pi / (g.nx * g.dx)
    n0 = 1.25
    pe = 0.4 + 0.05 * np.sin(k * x)
    E = O.ohm_pe(g, np.zeros((3, nc)), np.full(nc, n0), np.zeros((3, nc)), pe)
    assert np.abs(E[0] + 0.05 * np.cos(k * x) * math.sin(k * g.dx) / g.dx / n0).max() < 1e-14
    assert np.abs(E[1:]).max() == 0.0


# ----------------------------------------------------------------------------
# electrostatic model (Sec. 4, Eq. esohm; reading R17)
# ----------------------------------------------------------------------------

def es_grid(pe_eq=1, nsub=4):
    return O.make_grid(24, 1, 16, 0.5, 1.0, 0.5, 0.02, nsub=nsub, Te=0.1, gamma_e=GAM, eta=1e-3,
                       eta_h=1e-4, n_floor=0.05, shape="qs", pe_eq=pe_eq, kappa=0.0, ohm_model=1)


def test_electrostatic_ohm_keeps_only_the_pressure_gradient():
    """Whatever B and J_i are, E = -grad p_e / n_f."""
    g = es_grid()
    nc = g.nx * g.nz
    rng = np.random.default_rng(5)
    x, _ = centres(g)
    k = 2 * math.pi / (g.nx * g.dx)
    n0 = 1.4
    pe = 0.4 + 0.05 * np.sin(k * x)
    E = O.ohm_pe(g, rng.normal(size=(3, nc)), np.full(nc, n0), rng.normal(size=(3, nc)), pe)
    assert np.abs(E[0] + 0.05 * np.cos(k * x) * math.sin(k * g.dx) / g.dx / n0).max() < 1e-14
    assert np.abs(E[1:]).max() < 1e-15


def test_electrostatic_field_advance_keeps_B_and_moves_p_with_the_ions():
    """B is not advanced; u_e = J_i / n_f, whatever curl B is."""
    g = es_grid()
    nc = g.nx * g.nz
    rng = np.random.default_rng(6)
    x, _ = centres(g)
    k = 2 * math.pi * 2 / (g.nx * g.dx)
    u0, p0, dl = 0.8, 0.5, 0.01
    B = rng.normal(size=(3, nc))
    n = np.ones(nc)
    Ji = np.zeros((3, nc))
    Ji[0] = u0
    pe = p0 + dl * np.sin(k * x)
    h = g.dt / g.nsub
    lam = -1j * u0 * math.sin(k * g.dx) / g.dx
    G = (1 + lam * h + (lam * h) ** 2 / 2) ** g.nsub
    B1, p1 = O.field_advance_pe(g, B, pe, n, Ji)
    assert np.array_equal(B1, B)
    assert np.abs(p1 - (p0 + dl * np.imag(G * np.exp(1j * k * x)))).max() < 1e-14
    g0 = es_grid(pe_eq=0)
    assert np.array_equal(O.field_advance(g0, B, n, Ji), B)
