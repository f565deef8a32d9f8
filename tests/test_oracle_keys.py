"""The ion order the library documents (include/hv.h: sort_every, hv_query),
as restated by oracle.supercell_keys for the sort tests: pinned by hand
examples and invariants (no GPU)."""
import numpy as np

import oracle as O


def test_keys_without_prediction_are_the_cell_keys():
    # 8x1x8 cells, 4x1x4 tiles: tile (ti, tk) = (i // 4, k // 4), key =
    # tile * 16 + (i % 4) + 4 * (k % 4)
    cells = np.array([0, 3, 4, 9, 63])
    want = [0, 3, 16, 0 * 16 + 1 + 4 * 1, 3 * 16 + 3 + 4 * 3]
    assert list(O.supercell_keys(cells, 8, 1, 8, (4, 1, 4))) == want


def test_predicted_key_cells_by_hand():
    pc = (np.float32(0.32), np.float32(0.0), np.float32(0.32))
    off = np.array([[0.99, -0.5, 0.9, 0.5], [0, 0, 0, 0], [0, 0, 0.5, -0.9]], np.float32)
    v = np.array([[1.0, -9.0, 2.0, 0.0], [0, 0, 0, 0], [0, 0, 2.0, -1.0]], np.float32)
    cells = np.array([0, 5, 63, 8])
    keys = O.supercell_keys(cells, 8, 1, 8, (4, 1, 4), off=off, v=v, pc=pc)
    # 0.99 + 0.32 >= 1: cell 0 -> i = 1; -0.5 - 2.88 < -1: i 5 -> 4 (tile 1);
    # 0.9 + 0.64 and 0.5 + 0.64 >= 1: (7, 7) -> (0, 0) periodically;
    # z of cell 8 (i 0, k 1): -0.9 - 0.32 < -1 -> k 0
    assert list(keys) == [1, 16, 0, 0]


def test_predicted_key_cell_within_one_and_zero_pc_is_plain():
    rng = np.random.default_rng(3)
    nx, ny, nz, tile = 20, 6, 12, (8, 8, 8)
    n = 5000
    cells = rng.integers(0, nx * ny * nz, n)
    off = rng.uniform(-1, 1, (3, n)).astype(np.float32)
    v = rng.normal(0, 3, (3, n)).astype(np.float32)
    plain = O.supercell_keys(cells, nx, ny, nz, tile)
    zero = (np.float32(0),) * 3
    assert np.array_equal(O.supercell_keys(cells, nx, ny, nz, tile, off=off, v=v, pc=zero), plain)
    # invert keys to cells: the key cell is at most one cell from the ion's
    # cell per axis (periodically) and moves only where off + v pc leaves [-1, 1)
    pc = (np.float32(0.4), np.float32(0.4), np.float32(0.4))
    k = O.supercell_keys(cells, nx, ny, nz, tile, off=off, v=v, pc=pc)
    tx, ty, tz = tile
    ntx, nty = -(-nx // tx), -(-ny // ty)
    t, loc = k // (tx * ty * tz), k % (tx * ty * tz)
    ki = (t % ntx) * tx + loc % tx
    kj = ((t // ntx) % nty) * ty + (loc // tx) % ty
    kk = (t // (ntx * nty)) * tz + loc // (tx * ty)
    ci, cj, ck = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    for kc, c, m, a in ((ki, ci, nx, 0), (kj, cj, ny, 1), (kk, ck, nz, 2)):
        d = (kc - c + m + 1) % m - 1
        assert set(np.unique(d)) <= {-1, 0, 1}
        q = off[a].astype(np.float64) + v[a].astype(np.float64) * 0.4
        assert (d[np.abs(q) < 0.999] == 0).all()
        assert (d[q > 1.001] == 1).all() and (d[q < -1.001] == -1).all()


def test_prediction_coefficients():
    # 1.375 * sort_every * dt / Delta in FP32 per axis with more than one
    # cell; none without sorting or with open faces
    p = dict(nx=8, ny=1, nz=4, dx=0.25, dy=1.0, dz=0.5, dt=0.02, sort_every=8)
    pc = O.sort_pred_coeffs(p)
    assert pc == (np.float32(0.88), np.float32(0.0), np.float32(0.44))
    assert all(c == 0 for c in O.sort_pred_coeffs(dict(p, sort_every=0)))
    assert all(c == 0 for c in O.sort_pred_coeffs(dict(p, open_faces=1)))
