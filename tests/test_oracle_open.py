"""Pins of the oracle's open faces (Sec. 2.3; readings R21-R23): ghost cells
copy B1, B0 and the moments of their interior neighbour; Ohm's law in a
ghost cell drops the derivatives normal to the face and keeps the
tangential ones; deposits beyond a face fold onto the cell next to it;
ions leaving through an open face are removed.  Each pin fails for a
plausible mistake (a ghost filled periodically, a normal derivative kept,
the fold sent to the far side, an ion wrapped instead of absorbed)."""
import numpy as np

import oracle as O


def grid(nx, nz, open_axes=(1, 0, 0), **kw):
    p = dict(dx=0.5, dz=0.5, dt=0.01, nsub=4, Te=1.0, n_floor=0.01, shape="qs", eta=0.0,
             eta_h=0.0)
    p.update(kw)
    return O.make_grid(nx, 1, nz, p["dx"], 1.0, p["dz"], p["dt"], p["nsub"], p["Te"], 1.0,
                       p["eta"], p["eta_h"], p["n_floor"], p["shape"], open_axes=open_axes)


def ext(g, F):
    Nz, Ny, Nx = O.xshape(g)
    return np.asarray(F).reshape(-1, Nz, Ny, Nx)


def test_pressure_gradient_in_ghost_cells_has_no_normal_component():
    """n linear along the open x axis, uniform along z: E_x = -dp/dx / n in
    the interior (one-sided half difference next to the faces, where the
    ghost copies the neighbour), exactly zero in the ghost cells."""
    nx, nz, dx = 12, 6, 0.5
    g = grid(nx, nz)
    x = (np.arange(nx) + 0.5) * dx
    n = np.tile(1.0 + 0.1 * x, nz)
    B1 = np.zeros((3, nx * nz))
    E = ext(g, O.ohm_open(g, B1, n, np.zeros((3, nx * nz))))
    Ex = E[0][:, 0, :]  # [nz][nx + 2]
    assert np.all(Ex[:, 0] == 0.0) and np.all(Ex[:, -1] == 0.0)
    nn = 1.0 + 0.1 * x
    interior = -(np.roll(nn, -1) - np.roll(nn, 1)) / (2 * dx) / nn
    interior[0] = -(nn[1] - nn[0]) / (2 * dx) / nn[0]
    interior[-1] = -(nn[-1] - nn[-2]) / (2 * dx) / nn[-1]
    assert np.allclose(Ex[:, 1:-1], interior[None, :], rtol=1e-13, atol=0)
    assert np.abs(E[1]).max() == 0.0 and np.abs(E[2]).max() < 1e-15


def test_tangential_gradient_kept_in_ghost_cells():
    """n varies along the periodic z axis only: a ghost cell of the open x
    face has the same E_z = -dp/dz / n as its interior neighbour."""
    nx, nz, dz = 8, 10, 0.5
    g = grid(nx, nz)
    z = (np.arange(nz) + 0.5) * dz
    n = np.repeat(1.0 + 0.2 * np.sin(2 * np.pi * z / (nz * dz)), nx)
    E = ext(g, O.ohm_open(g, np.zeros((3, nx * nz)), n, np.zeros((3, nx * nz))))
    Ez = E[2][:, 0, :]
    assert np.abs(Ez).max() > 1e-3
    assert np.array_equal(Ez[:, 0], Ez[:, 1]) and np.array_equal(Ez[:, -1], Ez[:, -2])


def test_hall_term_in_ghost_cells_drops_the_normal_curl():
    """B1 = (1, f(x), 0) with x open: J_z = df/dx (centred; one-sided half
    next to a face) in the interior, zero in the ghost cells, so the ghost
    Hall field E = J x B / n vanishes there."""
    nx, nz, dx = 10, 4, 0.5
    g = grid(nx, nz, Te=0.0)
    x = (np.arange(nx) + 0.5) * dx
    f = 0.1 * x ** 2
    B1 = np.zeros((3, nx * nz))
    B1[0] = 1.0
    B1[1] = np.tile(f, nz)
    E = ext(g, O.ohm_open(g, B1, np.ones(nx * nz), np.zeros((3, nx * nz))))
    Jz = np.empty(nx)
    Jz[1:-1] = (f[2:] - f[:-2]) / (2 * dx)
    Jz[0], Jz[-1] = (f[1] - f[0]) / (2 * dx), (f[-1] - f[-2]) / (2 * dx)
    Ey = E[1][:, 0, :]
    assert np.all(Ey[:, 0] == 0.0) and np.all(Ey[:, -1] == 0.0)
    assert np.allclose(Ey[:, 1:-1], Jz[None, :] * 1.0, rtol=1e-13, atol=1e-15)  # E_y = J_z B_x


def test_x_invariant_state_advances_as_if_periodic():
    """Nothing varies along the open axis: the ghost copies equal the
    periodic images, so the open-face field advance equals the periodic one
    (a circularly polarised mode along z, Hall, resistive and
    hyper-resistive terms on)."""
    nx, nz, dz = 6, 32, 0.5
    kw = dict(Te=0.1, eta=1e-3, eta_h=1e-4)
    go, gp = grid(nx, nz, **kw), grid(nx, nz, open_axes=(0, 0, 0), **kw)
    z = np.repeat((np.arange(nz) + 0.5) * dz, nx)
    k = 2 * np.pi / (nz * dz)
    B1 = np.zeros((3, nx * nz))
    B1[2] = 1.0
    B1[0] = 0.05 * np.cos(k * z)
    B1[1] = 0.05 * np.sin(k * z)
    n = 1.0 + 0.1 * np.cos(k * z)
    Ji = np.zeros((3, nx * nz))
    Ji[0] = 0.02 * np.sin(k * z)
    a = O.field_advance_open(go, B1, n, Ji)
    b = O.field_advance(gp, B1, n, Ji)
    assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()


def test_deposit_beyond_an_open_face_folds_onto_the_boundary_cell():
    """One ion at the centre of the first cell of an open x axis (QS): the
    -x neighbour weight 1/12 lands on the cell itself (3/4 in total), not on
    the far side; charge equals q w."""
    nx, nz = 6, 4
    g = grid(nx, nz, dt=1e-6)
    c = 1 * nx + 0  # i = 0, k = 1
    sp = O.Species(1.0, 1.0, np.array([c]), np.zeros((3, 1)), np.zeros((3, 1)), np.array([0.25]))
    sim = O.Sim(g, [sp], np.vstack([np.ones(nx * nz), np.zeros(nx * nz), np.zeros(nx * nz)]))
    n = sim.n_prev.reshape(nz, nx)  # q w / V_c = 1 here, so n is the shape weight
    assert abs(n[1, 0] - 0.75) < 1e-15 and abs(n[1, 1] - 1.0 / 12) < 1e-15
    assert n[1, nx - 1] == 0.0  # nothing wrapped to the far side
    assert abs(n[0, 0] - 1.0 / 12) < 1e-15 and abs(n[2, 0] - 1.0 / 12) < 1e-15
    assert abs(sim.n_prev.sum() * 0.25 - 0.25) < 1e-15


def test_ions_leave_through_open_faces_and_wrap_through_periodic_ones():
    nx, nz = 6, 4
    g = grid(nx, nz, dt=0.1, Te=0.0)
    # four ions next to faces moving outwards: -x, +x (open), -z, +z (periodic)
    cells = np.array([1 * nx + 0, 2 * nx + nx - 1, 0 * nx + 3, (nz - 1) * nx + 2])
    off = np.zeros((3, 4))
    off[0] = [-0.9, 0.9, 0.0, 0.0]
    off[2] = [0.0, 0.0, -0.9, 0.9]
    v = np.zeros((3, 4))
    v[0] = [-1.0, 1.0, 0.0, 0.0]
    v[2] = [0.0, 0.0, -1.0, 1.0]
    w = np.array([0.1, 0.2, 0.3, 0.4])
    B = np.zeros((3, nx * nz))
    sim = O.Sim(g, [O.Species(1.0, 1e6, cells, off, v, w)], B)  # heavy: no field kicks
    sim.step(1)
    s = sim.species[0]
    assert s.n == 2 and np.array_equal(s.w, [0.3, 0.4])  # the x movers are gone
    assert s.cell[0] // nx == nz - 1 and s.cell[1] // nx == 0  # z movers wrapped
