"""The step's sort, bit-exact against the oracle's stable counting sort.

The library sorts every species by supercell key (tile index, then the cell
inside the tile) every sort_every steps, keeping the order of ions with
equal keys.  The key cell of an ion is its cell moved by at most one cell
along each axis toward where it is predicted to be 0.6875 sort intervals
later (off + v * 1.375 * sort_every * dt / Delta outside [-1, 1), FP32;
oracle.supercell_keys and oracle.sort_pred_coeffs restate it).  Ions are identified by distinct weights, which the library
copies bit for bit, so the order hv_get_ions reports after a step is the
sort's permutation applied to the order before it (the push moves ions
in place).  Each sort is checked against oracle.sort_stable on the keys of
the pre-sort cells:
  * the permutation: the post-sort weight sequence equals the pre-sort
    sequence gathered by the oracle's permutation (integer work: exact);
  * the tile ranges (hv_get_tile_offsets): the oracle's key offsets at the
    first key of every tile (exact).
The first sort after loading takes the general path (radix passes); later
sorts at most 8 (2D) or 2 (3D) steps after the previous one take the
windowed path, longer intervals the general path again.  The cases cover
ragged tiles, windows wider than the grid (two tiles per axis), a single
tile, two species and both paths in 2D and 3D."""
import numpy as np
import pytest

import oracle as O
from paper_2305_05600_gb300 import inputs as I

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


def two_species(wl):
    s = wl.species[0]
    h = s.n // 3
    cut = lambda a, sl: np.ascontiguousarray(a[..., sl])  # noqa: E731
    wl.species = [I.SpeciesInput(1.0, 1.0, cut(s.cell, slice(0, h)), cut(s.off, slice(0, h)),
                                 cut(s.v, slice(0, h)), cut(s.w, slice(0, h))),
                  I.SpeciesInput(1.0, 2.0, cut(s.cell, slice(h, None)),
                                 cut(s.off, slice(h, None)), cut(s.v, slice(h, None)),
                                 cut(s.w, slice(h, None)))]
    return I.with_distinct_weights(wl)


CASES = {
    # 2D, 40x24 cells (ragged tiles), windowed sorts every 2 steps
    "2d_ragged_every2": lambda: I.harris(nx=40, nz=24, ppc=24, dx=0.25, seed=41, sort_every=2),
    # 2D, 24x24 cells: every window is wider than the grid (two tiles per axis)
    "2d_wide_window_every8": lambda: I.harris(nx=24, nz=24, ppc=16, dx=0.25, seed=42,
                                              sort_every=8),
    # 2D single tile
    "2d_single_tile_every3": lambda: I.harris(nx=16, nz=16, ppc=16, dx=0.25, seed=43,
                                              sort_every=3),
    # 2D, longer than the window: every sort takes the general path
    "2d_general_every10": lambda: I.harris(nx=40, nz=24, ppc=24, dx=0.25, seed=44,
                                           sort_every=10),
    # 3D, ragged tiles, windowed sorts every 2 steps (fast beam ions)
    "3d_ragged_every2": lambda: I.beam3d(nx=12, ny=10, nz=9, n_core=6, n_beam=3, dx=0.5,
                                         seed=45, sort_every=2),
    # 3D, sort every 4 steps: the general path (the window holds 2 steps)
    "3d_ragged_every4": lambda: I.beam3d(nx=12, ny=10, nz=9, n_core=6, n_beam=3, dx=0.5,
                                         seed=51, sort_every=4),
    # 3D, sort every 20 steps: the general path
    "3d_general_every20": lambda: I.beam3d(nx=20, ny=17, nz=9, n_core=3, n_beam=1, dx=0.5,
                                           seed=46, sort_every=20),
    # two species sorted separately, 2D windowed
    "2d_two_species_every4": lambda: two_species(I.harris(nx=40, nz=24, ppc=12, dx=0.25,
                                                          seed=47, sort_every=4)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_step_sort_bit_exact(hvmod, case):
    wl = CASES[case]()
    if len(wl.species) == 1:
        wl = I.with_distinct_weights(wl)
    p = wl.params
    S = p["sort_every"]
    nsteps = 2 * S + 1  # the first sort (general path) and two more
    ctx = hvmod.load_workload(wl)
    tile = hvmod.hv_query(ctx)["tile"]
    nkeys = O.supercell_nkeys(p["nx"], p["ny"], p["nz"], tile)
    per_tile = tile[0] * tile[1] * tile[2]
    nsorts = 0
    before = [hvmod.hv_get_ions(ctx, s) for s in range(len(wl.species))]
    for step in range(nsteps):
        hvmod.hv_step(ctx, 1)
        after = [hvmod.hv_get_ions(ctx, s) for s in range(len(wl.species))]
        if step % S == 0:
            nsorts += 1
            for s in range(len(wl.species)):
                keys = O.supercell_keys(before[s]["cell"], p["nx"], p["ny"], p["nz"], tile,
                                        off=before[s]["off"], v=before[s]["v"],
                                        pc=O.sort_pred_coeffs(p))
                perm, counts, offsets = O.sort_stable(keys, nkeys)
                assert np.array_equal(after[s]["w"], before[s]["w"][perm]), (case, step, s)
                tile_off = hvmod.hv_get_tile_offsets(ctx, s)
                assert np.array_equal(tile_off.astype(np.int64), offsets[::per_tile]), (case, step)
                # and the ions are in key order now (the push moves them afterwards)
                assert counts.sum() == before[s]["w"].shape[0]
        else:
            for s in range(len(wl.species)):
                assert np.array_equal(after[s]["w"], before[s]["w"]), "no sort: order unchanged"
        before = after
    assert nsorts == 3
    d = hvmod.hv_diag(ctx)
    assert d["err_word"] == 0
    ctx.close()


def test_tile_offsets_before_the_first_sort(hvmod):
    """Before the first sort the tile ranges split the ions evenly."""
    wl = I.with_distinct_weights(I.harris(nx=40, nz=24, ppc=10, dx=0.25, seed=48, sort_every=0))
    ctx = hvmod.load_workload(wl)
    nt = hvmod.hv_query(ctx)["ntiles"]
    n = wl.n_particles
    want = (np.arange(nt + 1, dtype=np.int64) * n) // nt
    assert np.array_equal(hvmod.hv_get_tile_offsets(ctx, 0).astype(np.int64), want)
    hvmod.hv_step(ctx, 2)  # sort_every = 0: never sorted, order kept
    g = hvmod.hv_get_ions(ctx, 0)
    assert np.array_equal(g["w"], wl.species[0].w)
    ctx.close()


def test_injected_timeout_is_reported(hvmod):
    """The error path of a bounded device wait that gave up, without any
    wait running out: the error bit is injected on the host and the next
    synchronising call reports HV_ETIMEOUT."""
    wl = I.harris(nx=32, nz=16, ppc=4, dx=0.25, seed=49, sort_every=1)
    ctx = hvmod.load_workload(wl)
    hvmod.hv_step(ctx, 1)
    assert hvmod.hv_diag(ctx)["err_word"] == 0
    hvmod.hv_inject_error(ctx, 8)
    d = hvmod.hv_diag(ctx, check=False)
    assert d["status"] == hvmod.HV_ETIMEOUT and d["err_word"] == 8
    with pytest.raises(hvmod.HVError, match="HV_ETIMEOUT"):
        hvmod.hv_moments(ctx)
    ctx.close()
