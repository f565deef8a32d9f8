"""Open faces and injection (Sec. 2.3) on the GPU against the oracle.

* Without injection: a Harris-sheet box open in x (2D) and an ion-beam box
  open in x and z (3D) for three steps, sorted every 2 (the sort moves the
  slots of absorbed ions behind the live ones): the live ions (identified
  by distinct weights: both sides must have absorbed the same ions), the
  deposited moments, B, E and the diagnostics, with the step tolerances.
* With injection: a uniform plasma flowing through a box open in x, the same
  drifting Maxwellian injected at both faces every step (Philox words keyed
  by the seed), sorted every 3 steps; the live ions in library order, which
  both sides keep the same (survivors in order, injected ions appended in
  face-cell order, stable sorts), element by element.  The GPU inverts the
  flux-weighted speed distribution in FP32, which moves an injected speed
  by up to ~1e-6 (and more for the rare ions with a tiny inward speed), so
  injected velocities are bounded by 1e-4 (|v| + vt)."""
import numpy as np
import pytest

import oracle as O
from paper_2305_05600_gb300 import inputs as I
from tests.helpers import check_diagnostics, oracle_sim, periodic_delta, phys_pos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hvmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_05600_gb300 import hv
    hv.lib()
    hv.hv_set_allocator(True)
    return hv


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def key_fn(hvmod, ctx, p):
    tile = hvmod.hv_query(ctx)["tile"]
    return lambda cell: O.supercell_keys(cell, p["nx"], p["ny"], p["nz"], tile)


def compare_by_weight(p, g, sp, vscale):
    og = np.argsort(g["w"], kind="stable")
    oo = np.argsort(sp.w, kind="stable")
    assert np.array_equal(g["w"][og].astype(np.float64), sp.w[oo])
    d = periodic_delta(p, phys_pos(p, g["cell"][og], g["off"][:, og].astype(np.float64)),
                       phys_pos(p, sp.cell[oo], sp.off[:, oo]))
    dl = np.array([p["dx"], p["dy"], p["dz"]])[:, None]
    assert np.abs(d / dl).max() < 1e-5
    dv = np.abs(g["v"][:, og].astype(np.float64) - sp.v[:, oo])
    vmag = np.linalg.norm(sp.v[:, oo], axis=0)
    assert (dv.max(axis=0) <= 1e-5 * (vmag + vscale)).all(), dv.max()


@pytest.mark.parametrize("dim", [2, 3])
def test_open_faces_without_injection(hvmod, dim):
    if dim == 2:
        wl = I.harris(nx=40, nz=24, ppc=24, dx=0.25, seed=71, sort_every=2)
        wl.params["open_faces"] = 1
    else:
        wl = I.beam3d(nx=12, ny=10, nz=9, n_core=6, n_beam=3, dx=0.5, seed=72, sort_every=2)
        wl.params["open_faces"] = 1 | 4
    wl = I.with_distinct_weights(wl)
    p = wl.params
    ctx = hvmod.load_workload(wl)
    sim = oracle_sim(wl)
    vscale = float(np.sqrt(np.mean(wl.species[0].v.astype(np.float64) ** 2)))
    m0 = hvmod.hv_moments(ctx)
    assert rel_l2(m0["n"].reshape(-1), sim.n_prev) < 1e-5
    assert rel_l2(m0["E"].reshape(3, -1), sim.E) < 1e-4
    n0 = wl.species[0].n
    for _ in range(3):
        hvmod.hv_step(ctx, 1)
        sim.step(1, sort_every=p["sort_every"], key_fn=key_fn(hvmod, ctx, p))
        g = hvmod.hv_get_ions(ctx, 0)
        compare_by_weight(p, g, sim.species[0], vscale)
        m = hvmod.hv_moments(ctx)
        assert rel_l2(m["n"].reshape(-1), sim.n_prev) < 1e-5
        assert rel_l2(m["J"].reshape(3, -1), sim.J_prev) < 1e-5
        assert rel_l2(m["B"].reshape(3, -1), sim.B) < 1e-6
        assert rel_l2(m["E"].reshape(3, -1), sim.E) < 1e-4
        check_diagnostics(p, hvmod.hv_diag(ctx), sim, m["B"])
    assert sim.species[0].n < n0  # ions did leave through the open faces
    ctx.close()


def test_open_faces_with_injection(hvmod):
    wl = I.drifting_slab(nx=32, nz=16, ppc=16, U=0.6, Ti=0.04, seed=73, sort_every=3,
                         w_scale=1.0)
    wl = I.with_distinct_weights(wl)
    p = wl.params
    p["seed"] = 12345
    w_inj = 1.0 / 64.0  # exactly representable
    U, Ti = 0.6, 0.04
    faces = [(0, O.inject_face(0, 1.0, (U, 0, 0), Ti, w_inj)),
             (0, O.inject_face(1, 1.0, (U, 0, 0), Ti, w_inj))]
    ctx = hvmod.hv_init_grid(p, wl.B0)
    s = wl.species[0]
    hvmod.hv_load_ions(ctx, 0, s.q, s.m, s.cell, s.off, s.v, s.w)
    hvmod.hv_reserve_ions(ctx, 0, 2 * s.n)
    for face, f in faces:
        hvmod.hv_set_injection(ctx, 0, f.face, f.n, list(f.u), f.T, f.w)
    sim = oracle_sim(wl, inject=faces, seed=12345)
    vt = np.sqrt(Ti)
    for step in range(4):
        hvmod.hv_step(ctx, 1)
        sim.step(1, sort_every=p["sort_every"], key_fn=key_fn(hvmod, ctx, p))
        g = hvmod.hv_get_ions(ctx, 0)
        sp = sim.species[0]
        assert g["w"].shape[0] == sp.n, (step, g["w"].shape[0], sp.n)
        assert np.array_equal(g["w"].astype(np.float64), sp.w)
        d = periodic_delta(p, phys_pos(p, g["cell"], g["off"].astype(np.float64)),
                           phys_pos(p, sp.cell, sp.off))
        dl = np.array([p["dx"], p["dy"], p["dz"]])[:, None]
        assert np.abs(d / dl).max() < 1e-4
        dv = np.abs(g["v"].astype(np.float64) - sp.v)
        vmag = np.linalg.norm(sp.v, axis=0)
        assert (dv.max(axis=0) <= 1e-4 * (vmag + vt)).all(), dv.max()
        m = hvmod.hv_moments(ctx)
        assert rel_l2(m["n"].reshape(-1), sim.n_prev) < 1e-5
        assert rel_l2(m["B"].reshape(3, -1), sim.B) < 1e-6
        dg = hvmod.hv_diag(ctx)
        od = sim.diags[-1]
        assert abs(dg["charge"] - od["charge"]) < 1e-5 * od["charge"]
    # ions did enter: about 0.38 per face cell and step at the inflow face
    assert (sim.species[0].w == w_inj).sum() > 15
    ctx.close()
