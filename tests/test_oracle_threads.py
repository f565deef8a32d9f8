"""The oracle's all-core mode (the CPU baseline on every host core) against
its one-thread mode, which is the parity reference: particles split into
contiguous ranges with private deposit grids added in thread order, and
cell loops that write one value per cell, must give the same step up to
FP64 summation order (1e-12 relative); after the first step (same fields)
the particles are identical, later they differ by the fields' rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2305_05600_gb300 import inputs as I
from tests.helpers import oracle_sim


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim", [2, 3])
def test_threaded_oracle_matches_one_thread(dim):
    if dim == 2:
        wl = I.harris(nx=32, nz=16, ppc=20, dx=0.25, seed=61, sort_every=0)
    else:
        wl = I.beam3d(nx=8, ny=6, nz=5, n_core=6, n_beam=2, dx=0.5, seed=62, sort_every=0)
    try:
        O.set_threads(1)
        a = oracle_sim(wl)
        a.step(1)
        O.set_threads(4)
        b = oracle_sim(wl)
        b.step(1)
        sa, sb = a.species[0], b.species[0]
        assert np.array_equal(sa.cell, sb.cell)
        assert np.array_equal(sa.off, sb.off) and np.array_equal(sa.v, sb.v)
        O.set_threads(1)
        a.step(2)
        O.set_threads(4)
        b.step(2)
    finally:
        O.set_threads(1)
    sa, sb = a.species[0], b.species[0]
    assert rel(sb.v, sa.v) < 1e-12 and rel(sb.off, sa.off) < 1e-12
    assert rel(b.n_prev, a.n_prev) < 1e-12
    assert rel(b.J_prev, a.J_prev) < 1e-12
    assert rel(b.B, a.B) < 1e-12
    assert rel(b.E, a.E) < 1e-12
    for k in ("W_K", "W_B", "charge"):
        assert abs(b.diags[-1][k] - a.diags[-1][k]) <= 1e-12 * abs(a.diags[-1][k])
