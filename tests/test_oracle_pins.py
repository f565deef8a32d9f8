"""Pins of the FP64 oracle against what the paper and the mathematics fix:
closed forms, invariants, an independent formula from the paper (the QS
interpolation-coefficient form of App. B, Eqs. 18-19), brute force on tiny
grids and library special cases.  Each test is chosen so that a plausible
mistake (a dropped term, a wrong sign or index, a transposed operand) in the
oracle fails it.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(12345)


def grid(nx=4, ny=4, nz=4, dx=1.0, dy=1.0, dz=1.0, dt=0.1, **kw):
    return O.make_grid(nx, ny, nz, dx, dy, dz, dt, **kw)


def cidx(g, i, j, k):
    return (i % g.nx) + g.nx * ((j % g.ny) + g.ny * (k % g.nz))


# ----------------------------------------------------------------------------
# Boris push (Sec. 2.2, Eq. 9)
# ----------------------------------------------------------------------------

def test_boris_speed_conserved_in_pure_B():
    for _ in range(20):
        B = RNG.normal(size=3) * 3.0
        v = RNG.normal(size=3)
        s0 = np.linalg.norm(v)
        for _ in range(500):
            v = O.boris(0.37, [0, 0, 0], B, v)
        assert abs(np.linalg.norm(v) - s0) < 1e-12 * s0


@pytest.mark.parametrize("om_dt", [0.01, 0.3, 1.7])
def test_boris_gyrophase_is_2atan(om_dt):
    """Per step the Boris rotation turns v by 2 atan(Omega dt / 2) exactly, in
    the ion (left-hand) sense about B; the phase error against Omega N dt is
    the closed form 2N atan(Omega dt/2) - N Omega dt."""
    Bz = 2.0
    qmdt = om_dt / Bz
    v = np.array([1.0, 0.0, 0.0])
    N = 37
    for _ in range(N):
        v = O.boris(qmdt, [0, 0, 0], [0, 0, Bz], v)
    ang = math.atan2(v[1], v[0])
    expect = -N * 2.0 * math.atan(om_dt / 2.0)
    diff = (ang - expect + math.pi) % (2 * math.pi) - math.pi
    assert abs(diff) < 1e-12
    assert abs(v[2]) < 1e-15


def test_exb_drift_is_fixed_point_and_gyration_conserved():
    E = np.array([0.3, -0.2, 0.5])
    B = np.array([0.4, 1.1, -0.7])
    vE = np.cross(E, B) / B.dot(B)
    # E parallel to B accelerates along B; remove it for a pure E x B drift
    Eperp = E - E.dot(B) / B.dot(B) * B
    v = vE.copy()
    for _ in range(200):
        v = O.boris(0.05, Eperp, B, v)
    assert np.allclose(v, vE, atol=1e-13)
    # from rest: |v - v_E| is conserved (rotation about B around the drift)
    v = np.zeros(3)
    r0 = np.linalg.norm(v - vE)
    for _ in range(300):
        v = O.boris(0.05, Eperp, B, v)
        assert abs(np.linalg.norm(v - vE) - r0) < 1e-12


def test_boris_parallel_E_accelerates_linearly():
    B = np.array([0.0, 0.0, 1.5])
    E = np.array([0.0, 0.0, 0.2])
    v = np.zeros(3)
    for _ in range(10):
        v = O.boris(0.1, E, B, v)
    assert np.allclose(v, [0, 0, 10 * 0.1 * 0.2], atol=1e-15)


# ----------------------------------------------------------------------------
# Move (Sec. 2.2, Eq. 10) against a brute-force physical-coordinate update
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 1, 3)])
def test_move_brute_force(dims):
    nx, ny, nz = dims
    g = grid(nx, ny, nz, dx=0.7, dy=1.3, dz=0.4, dt=0.25)
    L = np.array([nx * 0.7, ny * 1.3, nz * 0.4])
    dl = np.array([0.7, 1.3, 0.4])
    n = np.array(dims)
    for _ in range(400):
        cell = int(RNG.integers(0, nx * ny * nz))
        d = RNG.uniform(-1, 1, 3)
        d[n == 1] = 0.0
        v = RNG.normal(size=3) * 3.0
        i = np.array([cell % nx, (cell // nx) % ny, cell // (nx * ny)])
        x = (i + 0.5 + 0.5 * d) * dl
        xn = x + v * g.dt
        c2, d2 = O.move(g, cell, d, v, 1.0)
        for a in range(3):
            if n[a] == 1:
                assert d2[a] == d[a]
                continue
            xa = xn[a] % L[a]
            ia = math.floor(xa / dl[a])
            oa = 2.0 * (xa / dl[a] - ia) - 1.0
            ja = [c2 % nx, (c2 // nx) % ny, c2 // (nx * ny)][a]
            got = (ja + 0.5 + 0.5 * d2[a]) * dl[a]
            dd = (got - xa + 0.5 * L[a]) % L[a] - 0.5 * L[a]
            assert abs(dd) < 1e-12
            assert -1.0 <= d2[a] < 1.0
            if abs(oa) < 1 - 1e-9:
                assert ja == ia % n[a]


def test_move_tie_goes_to_next_cell():
    g = grid(4, 1, 1, dt=1.0)
    # d + 2 v dt / dx = 1 exactly -> next cell with d = -1
    c, d = O.move(g, 1, [0.5, 0, 0], [0.25, 0, 0], 1.0)
    assert c == 2 and d[0] == -1.0


# ----------------------------------------------------------------------------
# Shapes: NGP (Eq. 13), QS (Eqs. 17-19), CIC (tensor-linear)
# ----------------------------------------------------------------------------

def _random_species(g, n, q=1.3, m=2.0):
    ncell = g.nx * g.ny * g.nz
    off = RNG.uniform(-1, 1, (3, n))
    for a, na in enumerate((g.nx, g.ny, g.nz)):
        if na == 1:
            off[a] = 0.0
    return O.Species(q, m, RNG.integers(0, ncell, n), off, RNG.normal(size=(3, n)),
                     RNG.uniform(0.5, 2.0, n))


@pytest.mark.parametrize("shape", ["ngp", "qs", "cic"])
@pytest.mark.parametrize("dims", [(4, 4, 4), (6, 1, 5)])
def test_deposit_total_charge_equals_sum_qw(shape, dims):
    g = grid(*dims, dx=0.5, dy=0.7 if dims[1] > 1 else 1.0, dz=0.3, shape=shape)
    sp = _random_species(g, 300)
    n, J = O.deposit(g, [sp])
    vc = g.dx * g.dy * g.dz
    assert abs(n.sum() * vc - sp.q * sp.w.sum()) < 1e-13 * sp.q * sp.w.sum()
    # current: sum J V_c = sum q w v
    for a in range(3):
        ref = (sp.q * sp.w * sp.v[a]).sum()
        assert abs(J[a].sum() * vc - ref) < 1e-12 * (abs(sp.q * sp.w).sum())


def test_weights_sum_to_one_and_are_nonnegative():
    for shape in ("ngp", "qs", "cic"):
        for _ in range(200):
            d = RNG.uniform(-1, 1, 3)
            _, wt = O.shape_weights(shape, d)
            assert abs(wt.sum() - 1.0) < 1e-15
            assert (wt >= 0).all()


def test_ngp_deposits_only_own_cell():
    g = grid(5, 4, 3, shape="ngp")
    sp = _random_species(g, 50)
    n, _ = O.deposit(g, [sp])
    ref = np.zeros(g.nx * g.ny * g.nz)
    np.add.at(ref, sp.cell, sp.q * sp.w)
    assert np.allclose(n, ref, rtol=0, atol=1e-14)


def test_cic_brute_force_hat_functions():
    """CIC deposit equals, for every cell, prod_a max(0, 1 - |x_p - X_c|_a /
    Delta_a) with minimum-image distances: a formula independent of the
    oracle's own-cell/side-neighbour stencil."""
    for dims in ((4, 4, 4), (4, 1, 4), (3, 3, 3)):
        g = grid(*dims, dx=0.5, dy=0.8 if dims[1] > 1 else 1.0, dz=0.6, shape="cic")
        sp = _random_species(g, 40)
        n, _ = O.deposit(g, [sp])
        nx, ny, nz = dims
        dl = np.array([g.dx, g.dy, g.dz])
        L = np.array(dims) * dl
        ref = np.zeros(nx * ny * nz)
        vc = g.dx * g.dy * g.dz
        for p in range(sp.n):
            c = sp.cell[p]
            ip = np.array([c % nx, (c // nx) % ny, c // (nx * ny)])
            xp = (ip + 0.5 + 0.5 * sp.off[:, p]) * dl
            for cc in range(nx * ny * nz):
                ic = np.array([cc % nx, (cc // nx) % ny, cc // (nx * ny)])
                Xc = (ic + 0.5) * dl
                dd = xp - Xc
                dd = dd - L * np.round(dd / L)
                wgt = 1.0
                for a in range(3):
                    if dims[a] == 1:
                        continue  # single-cell axis: everything folds here
                    wgt *= max(0.0, 1.0 - abs(dd[a]) / dl[a])
                ref[cc] += sp.q * sp.w[p] * wgt / vc
        assert np.allclose(n, ref, rtol=1e-12, atol=1e-13)


def _qs_eq18_19(F, g, cell, d):
    """Field at a particle from the QS interpolation coefficients, written out
    from App. B Eq. 18 (F^0, F^x, F^y, F^z, F^xx, F^yy, F^zz) and Eq. 19."""
    i, j, k = cell % g.nx, (cell // g.nx) % g.ny, cell // (g.nx * g.ny)

    def f(a, b, c):
        return F[cidx(g, i + a, j + b, k + c)]

    F0 = (6 * f(0, 0, 0) + f(1, 0, 0) + f(0, 1, 0) + f(0, 0, 1) + f(-1, 0, 0) + f(0, -1, 0)
          + f(0, 0, -1)) / 12.0
    Fx = (f(1, 0, 0) - f(-1, 0, 0)) / 6.0
    Fy = (f(0, 1, 0) - f(0, -1, 0)) / 6.0
    Fz = (f(0, 0, 1) - f(0, 0, -1)) / 6.0
    Fxx = (f(1, 0, 0) + f(-1, 0, 0) - 2 * f(0, 0, 0)) / 12.0
    Fyy = (f(0, 1, 0) + f(0, -1, 0) - 2 * f(0, 0, 0)) / 12.0
    Fzz = (f(0, 0, 1) + f(0, 0, -1) - 2 * f(0, 0, 0)) / 12.0
    dx, dy, dz = d
    return F0 + dx * (Fx + dx * Fxx) + dy * (Fy + dy * Fyy) + dz * (Fz + dz * Fzz)


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 1, 4), (3, 4, 5)])
def test_qs_gather_matches_interpolation_coefficient_form(dims):
    g = grid(*dims, shape="qs")
    ncell = g.nx * g.ny * g.nz
    for _ in range(60):
        F = RNG.normal(size=ncell)
        cell = int(RNG.integers(0, ncell))
        d = RNG.uniform(-1, 1, 3)
        if dims[1] == 1:
            d[1] = 0.0
        got = O.gather(g, F, cell, d)[0]
        ref = _qs_eq18_19(F, g, cell, d)
        assert abs(got - ref) < 1e-13


@pytest.mark.parametrize("shape", ["ngp", "qs", "cic"])
def test_deposit_is_transpose_of_gather(shape):
    """<F, deposit(p)> V_c = q w F(x_p): the deposit and the gather use the same
    weights (App. B: consistent, free of self-forces).  With the previous test
    this pins the QS deposit (Eq. 17) to the interpolation form (Eq. 19)."""
    g = grid(4, 3, 5, dx=0.5, dy=0.7, dz=0.9, shape=shape)
    ncell = g.nx * g.ny * g.nz
    vc = g.dx * g.dy * g.dz
    for _ in range(40):
        sp = _random_species(g, 1)
        F = RNG.normal(size=ncell)
        n, _ = O.deposit(g, [sp])
        lhs = (F * n).sum() * vc
        rhs = sp.q * sp.w[0] * O.gather(g, F, sp.cell[0], sp.off[:, 0])[0]
        assert abs(lhs - rhs) < 1e-12


def _face_pair(g, axis, d, c):
    """The same physical point seen from cell c (d[axis] = +1) and from its
    upper neighbour along `axis` (d[axis] = -1)."""
    i, j, k = c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)
    sh = [0, 0, 0]
    sh[axis] = 1
    c2 = cidx(g, i + sh[0], j + sh[1], k + sh[2])
    d1 = d.copy()
    d1[axis] = 1.0
    d2 = d.copy()
    d2[axis] = -1.0
    s1 = O.Species(1.0, 1.0, [c], d1.reshape(3, 1), np.zeros((3, 1)), [1.0])
    s2 = O.Species(1.0, 1.0, [c2], d2.reshape(3, 1), np.zeros((3, 1)), [1.0])
    return c2, O.deposit(g, [s1])[0], O.deposit(g, [s2])[0]


def test_cic_assignment_continuous_across_cell_faces():
    """CIC is continuous in the particle position: a point on the upper face
    of cell i deposits identically seen from cell i (d = +1) and from cell i+1
    (d = -1)."""
    g = grid(5, 4, 4, shape="cic")
    for axis in range(3):
        for _ in range(20):
            c = int(RNG.integers(0, 80))
            _, n1, n2 = _face_pair(g, axis, RNG.uniform(-1, 1, 3), c)
            assert np.allclose(n1, n2, atol=1e-15)


def test_qs_face_weights_along_the_crossing_axis():
    """QS is not continuous across faces (App. B / Sec. 2.2: it lacks the
    continuity of a tensor-product spline; the transverse neighbours switch
    from cell i's to cell i+1's).  With zero transverse offsets the two cells
    on either side of the face still get 1/3 each from both sides; a swapped
    (1 +- dx)^2 assignment would break this."""
    g = grid(5, 4, 4, shape="qs")
    for axis in range(3):
        for _ in range(10):
            c = int(RNG.integers(0, 80))
            c2, n1, n2 = _face_pair(g, axis, np.zeros(3), c)
            for cc in (c, c2):
                assert abs(n1[cc] - 1.0 / 3.0) < 1e-15
                assert abs(n2[cc] - 1.0 / 3.0) < 1e-15


def test_qs_2d_folding_centre_weight():
    """On a single-cell y axis the QS y-neighbours fold onto the cell: centre
    weight (4 - dx^2 - dz^2)/6 regardless of dy."""
    g = grid(5, 1, 5, shape="qs")
    for _ in range(20):
        d = RNG.uniform(-1, 1, 3)
        s = O.Species(1.0, 1.0, [12], d.reshape(3, 1), np.zeros((3, 1)), [1.0])
        n, _ = O.deposit(g, [s])
        assert abs(n[12] - (4 - d[0] ** 2 - d[2] ** 2) / 6.0) < 1e-15


# ----------------------------------------------------------------------------
# Grid operators (Eq. 12) by Fourier eigen-checks
# ----------------------------------------------------------------------------

def _coords(g):
    c = np.arange(g.nx * g.ny * g.nz)
    i, j, k = c % g.nx, (c // g.nx) % g.ny, c // (g.nx * g.ny)
    return (i + 0.5) * g.dx, (j + 0.5) * g.dy, (k + 0.5) * g.dz


def test_centred_derivative_eigenvalue():
    """grad_c exp(i k x) = i sin(k dx)/dx exp(i k x) on the periodic grid."""
    g = grid(8, 6, 10, dx=0.3, dy=0.5, dz=0.2)
    x, y, z = _coords(g)
    for (mx, my, mz) in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 1, 4)]:
        kx, ky, kz = 2 * np.pi * mx / (8 * 0.3), 2 * np.pi * my / (6 * 0.5), 2 * np.pi * mz / (10 * 0.2)
        ph = kx * x + ky * y + kz * z
        gr = O.grad(g, np.sin(ph))
        keff = [math.sin(kx * 0.3) / 0.3, math.sin(ky * 0.5) / 0.5, math.sin(kz * 0.2) / 0.2]
        for a in range(3):
            assert np.allclose(gr[a], keff[a] * np.cos(ph), atol=1e-12)
        lp = O.lap(g, np.sin(ph), 1)[0]
        lam = sum(-(4 / h ** 2) * math.sin(kk * h / 2) ** 2
                  for kk, h in ((kx, 0.3), (ky, 0.5), (kz, 0.2)))
        assert np.allclose(lp, lam * np.sin(ph), atol=1e-11)


def test_curl_closed_form_and_div_curl_zero():
    g = grid(8, 6, 10, dx=0.3, dy=0.5, dz=0.2)
    x, y, z = _coords(g)
    kx, kz = 2 * np.pi / (8 * 0.3), 2 * np.pi * 2 / (10 * 0.2)
    # A = (0, sin(kx x + kz z), 0): curl A = (-d_z A_y, 0, d_x A_y)
    ph = kx * x + kz * z
    A = np.stack([np.zeros_like(x), np.sin(ph), np.zeros_like(x)])
    cA = O.curl(g, A)
    kxe, kze = math.sin(kx * 0.3) / 0.3, math.sin(kz * 0.2) / 0.2
    assert np.allclose(cA[0], -kze * np.cos(ph), atol=1e-12)
    assert np.allclose(cA[1], 0.0, atol=1e-12)
    assert np.allclose(cA[2], kxe * np.cos(ph), atol=1e-12)
    # div curl == 0 for an arbitrary field
    R = RNG.normal(size=(3, g.nx * g.ny * g.nz))
    assert np.abs(O.div(g, O.curl(g, R))).max() < 1e-12


# ----------------------------------------------------------------------------
# Ohm's law (Eqs. 2-4, 6 and the density floor)
# ----------------------------------------------------------------------------

def _ohm_grid(**kw):
    base = dict(nx=16, ny=1, nz=8, dx=0.5, dy=1.0, dz=0.5, dt=0.1, Te=0.3, eta=0.0,
                eta_h=0.0, n_floor=0.05)
    base.update(kw)
    return grid(**base)


def test_ohm_uniform_plasma_gives_zero_field():
    g = _ohm_grid(eta=0.1, eta_h=0.01)
    nc = g.nx * g.ny * g.nz
    B = np.tile(np.array([[0.3], [1.0], [-0.4]]), (1, nc))
    E = O.ohm(g, B, np.full(nc, 1.7), np.zeros((3, nc)))
    assert np.abs(E).max() == 0.0


def test_ohm_ion_flow_gives_motional_field():
    """Uniform n, B and ion current: E = -u_i x B."""
    g = _ohm_grid()
    nc = g.nx * g.ny * g.nz
    b = np.array([0.3, 1.0, -0.4])
    u = np.array([0.2, -0.1, 0.5])
    n = 2.0
    E = O.ohm(g, np.tile(b[:, None], (1, nc)), np.full(nc, n), np.tile((n * u)[:, None], (1, nc)))
    assert np.allclose(E, np.tile(-np.cross(u, b)[:, None], (1, nc)), atol=1e-15)


def test_ohm_hall_and_resistive_terms_single_mode():
    """B = (B0, db sin(k x), 0), n = n0, J_i = 0: J = curl_c B = (0, 0, db k_eff
    cos kx); E = J x B / n0 + eta J - eta_H lap J with lap eigenvalue
    -(4/dx^2) sin^2(k dx/2)."""
    g = _ohm_grid(eta=0.07, eta_h=0.02)
    nc = g.nx * g.ny * g.nz
    x, _, _ = _coords(g)
    k = 2 * np.pi * 2 / (g.nx * g.dx)
    keff = math.sin(k * g.dx) / g.dx
    lam = -(4 / g.dx ** 2) * math.sin(k * g.dx / 2) ** 2
    B0, db, n0 = 1.2, 0.05, 0.8
    B = np.stack([np.full(nc, B0), db * np.sin(k * x), np.zeros(nc)])
    E = O.ohm(g, B, np.full(nc, n0), np.zeros((3, nc)))
    Jz = db * keff * np.cos(k * x)
    # J x B with J = (0,0,Jz): (Jy Bz - Jz By, Jz Bx - Jx Bz, ...) = (-Jz By, Jz Bx, 0)
    Ex = -Jz * B[1] / n0
    Ey = Jz * B0 / n0
    Ez = 0.07 * Jz - 0.02 * lam * Jz
    assert np.allclose(E[0], Ex, atol=1e-14)
    assert np.allclose(E[1], Ey, atol=1e-14)
    assert np.allclose(E[2], Ez, atol=1e-14)


def test_ohm_pressure_gradient_and_floor():
    """n = n0 + dn sin(kx), uniform B, J_i = 0, isothermal: E_x = -Te
    d_x^c n / max(n, n_floor); below the floor the gradient of the floored
    pressure is used."""
    g = _ohm_grid(Te=0.4, n_floor=0.5)
    nc = g.nx * g.ny * g.nz
    x, _, _ = _coords(g)
    k = 2 * np.pi / (g.nx * g.dx)
    n = 1.0 + 0.8 * np.sin(k * x)  # dips below the floor 0.5
    B = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, nc))
    E = O.ohm(g, B, n, np.zeros((3, nc)))
    nf = np.maximum(n, 0.5)
    i = np.arange(nc) % g.nx
    k_ = np.arange(nc) // g.nx
    ip = (i + 1) % g.nx + g.nx * k_
    im = (i - 1) % g.nx + g.nx * k_
    ref = -0.4 * (nf[ip] - nf[im]) / (2 * g.dx) / nf
    assert np.allclose(E[0], ref, atol=1e-14)
    # where the floor is inactive on all three points this is the smooth formula
    ok = (n[ip] > 0.5) & (n[im] > 0.5) & (n > 0.5)
    keff = math.sin(k * g.dx) / g.dx
    assert np.allclose(E[0][ok], (-0.4 * 0.8 * keff * np.cos(k * x) / n)[ok], atol=1e-14)
    assert np.abs(E[1]).max() < 1e-15


def test_ohm_adiabatic_equation_of_state():
    g = _ohm_grid(Te=0.4, gamma_e=5.0 / 3.0, n_floor=0.0)
    nc = g.nx * g.ny * g.nz
    x, _, _ = _coords(g)
    k = 2 * np.pi / (g.nx * g.dx)
    n = 1.0 + 0.3 * np.sin(k * x)
    B = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, nc))
    E = O.ohm(g, B, n, np.zeros((3, nc)))
    pe = 0.4 * n ** (5.0 / 3.0)
    i = np.arange(nc) % g.nx
    kk = np.arange(nc) // g.nx
    ref = -(pe[(i + 1) % g.nx + g.nx * kk] - pe[(i - 1) % g.nx + g.nx * kk]) / (2 * g.dx) / n
    assert np.allclose(E[0], ref, atol=1e-14)


# ----------------------------------------------------------------------------
# Faraday subcycle (Eq. 5): field-only circularly polarised whistler
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("sign", [1, -1])
def test_subcycle_whistler_rk2_amplification(sign):
    """Immobile ions (J_i = 0), n = 1, B = B0 x^ + db (0, cos kx, s sin kx).
    curl_c b = -s k_eff b, so J x b = 0 and the system is exactly linear:
    E = J x B = -s k_eff B0 (b x x^) and d(b_y + i b_z)/dt = i k_eff^2 B0
    (b_y + i b_z): the perturbation rotates in the right-hand (electron)
    sense about B0 for either propagation direction.  Each explicit-midpoint
    substep multiplies b_y + i b_z by G = 1 + i w h - (w h)^2/2, w = k_eff^2 B0."""
    g = grid(32, 1, 1, dx=0.25, dt=0.02, nsub=4, Te=0.0)
    nc = 32
    x = (np.arange(nc) + 0.5) * 0.25
    k = 2 * np.pi * 3 / (32 * 0.25)
    keff = math.sin(k * 0.25) / 0.25
    B0, db = 1.3, 1e-3
    B = np.stack([np.full(nc, B0), db * np.cos(k * x), sign * db * np.sin(k * x)])
    Bn = O.field_advance(g, B, np.ones(nc), np.zeros((3, nc)))
    h = 0.02 / 4
    w = keff ** 2 * B0
    G = 1 + 1j * w * h - (w * h) ** 2 / 2
    a0 = (B[1] + 1j * B[2]) / (db * np.exp(1j * sign * k * x))
    a1 = (Bn[1] + 1j * Bn[2]) / (db * np.exp(1j * sign * k * x))
    assert np.allclose(a0, 1.0)
    assert np.allclose(a1, G ** 4, atol=1e-11)
    assert np.allclose(Bn[0], B0, atol=1e-15)


def test_whistler_cfl_instability_above_bound():
    """Sec. 2.1 whistler limit Omega dt < dx^2/pi: grid-scale noise stays
    bounded below it and blows up well above it."""
    nc = 32
    rng = np.random.default_rng(7)
    noise = 1e-6 * rng.normal(size=(3, nc))
    noise[0] = 0.0
    B = noise.copy()
    B[0] += 1.0
    dx = 0.25
    bound = dx * dx / math.pi
    g_ok = grid(nc, 1, 1, dx=dx, dt=0.5 * bound * 50, nsub=50)
    g_bad = grid(nc, 1, 1, dx=dx, dt=8.0 * bound * 10, nsub=10)
    Bo = O.field_advance(g_ok, B, np.ones(nc), np.zeros((3, nc)))
    Bb = O.field_advance(g_bad, B, np.ones(nc), np.zeros((3, nc)))
    amp0 = np.abs(noise[1:]).max()
    assert np.abs(Bo[1:]).max() < 2 * amp0
    assert np.abs(Bb[1:]).max() > 1e3 * amp0


# ----------------------------------------------------------------------------
# Extrapolation (Eq. 11) and smoothing
# ----------------------------------------------------------------------------

def test_extrapolation_constant_and_linear():
    a = RNG.normal(size=50)
    assert np.allclose(O.extrapolate(a, a), a, rtol=4e-16, atol=0)
    b = RNG.normal(size=50)
    # J(t) = a + b t sampled at t = -1/2 and t = 1/2, extrapolated to t = 1
    assert np.allclose(O.extrapolate(a + 0.5 * b, a - 0.5 * b), a + b, atol=1e-15)


def test_binomial_smoothing_fourier_attenuation():
    """One (1/4,1/2,1/4) pass per axis multiplies a Fourier mode by
    cos^2(k dx/2) per axis and conserves the sum."""
    g = grid(16, 1, 8, dx=0.5, dz=0.5)
    x, _, z = _coords(g)
    kx, kz = 2 * np.pi * 3 / 8.0, 2 * np.pi / 4.0
    f = np.cos(kx * x + kz * z)
    s = O.smooth(g, f, 2)
    fac = (math.cos(kx * 0.5 / 2) ** 2 * math.cos(kz * 0.5 / 2) ** 2) ** 2
    assert np.allclose(s, fac * f, atol=1e-14)
    r = RNG.normal(size=128)
    assert abs(O.smooth(g, r, 3).sum() - r.sum()) < 1e-12


# ----------------------------------------------------------------------------
# Sort: stable counting sort special case of a library stable sort
# ----------------------------------------------------------------------------

def test_sort_matches_numpy_stable_argsort():
    for n, nk in ((0, 5), (1, 1), (1000, 7), (5000, 300), (777, 4096)):
        keys = RNG.integers(0, nk, n)
        perm, counts, offs = O.sort_stable(keys, nk)
        assert np.array_equal(perm, np.argsort(keys, kind="stable"))
        assert np.array_equal(counts, np.bincount(keys, minlength=nk))
        assert offs[0] == 0 and np.array_equal(np.diff(offs), counts)


# ----------------------------------------------------------------------------
# Whole step invariants
# ----------------------------------------------------------------------------

def test_step_charge_and_divB_invariants():
    """Deposited charge equals sum q w every step; the discrete div B field is
    unchanged by the subcycled Faraday update (centred div of centred curl is
    zero), so it stays at its initial value (here the float32 rounding of the
    loaded B) to FP64 roundoff."""
    from paper_2305_05600_gb300 import inputs as I
    from tests.helpers import oracle_sim
    wl = I.harris(nx=32, nz=32, ppc=16, dx=0.25)
    sim = oracle_sim(wl)
    div0 = O.div(sim.g, sim.B)
    qw = sum((s.q * s.w.astype(np.float64)).sum() for s in wl.species)
    for _ in range(3):
        d = sim.step(1)
        assert abs(d["charge"] - qw) < 1e-12 * qw
        assert np.abs(O.div(sim.g, sim.B) - div0).max() < 1e-11
        assert abs(d["max_divB"] - np.abs(div0).max()) < 1e-11


def test_half_step_deposit_position_ngp():
    """NGP deposit lands in the cell containing x^n + v^{n+1/2} dt / 2."""
    g = grid(8, 1, 8, dx=0.5, dz=0.5, dt=0.2, shape="ngp")
    nc = 64
    for _ in range(50):
        c = int(RNG.integers(0, nc))
        d = RNG.uniform(-1, 1, 3)
        d[1] = 0
        v = RNG.normal(size=3) * 2
        sp = O.Species(1.0, 1.0, [c], d.reshape(3, 1), v.reshape(3, 1), [1.0])
        n, _, _ = O.push_deposit(g, [sp], np.zeros((3, nc)), np.zeros((3, nc)))
        i, k = c % 8, c // 8
        xh = (i + 0.5 + 0.5 * d[0]) * 0.5 + v[0] * 0.1
        zh = (k + 0.5 + 0.5 * d[2]) * 0.5 + v[2] * 0.1
        ih, kh = int(math.floor(xh / 0.5)) % 8, int(math.floor(zh / 0.5)) % 8
        fx, fz = (xh / 0.5) % 1.0, (zh / 0.5) % 1.0
        if min(fx, 1 - fx, fz, 1 - fz) < 1e-9:
            continue
        assert n[ih + 8 * kh] == pytest.approx(1.0 / 0.25)
