"""The oracle's QS deposit weights against the golden fixture
tests/golden/qs_eq17.txt: Eq. 17 (App. B) evaluated in exact rational
arithmetic at rational relative coordinates by tests/golden/make_qs_eq17.py,
which uses neither the oracle nor the library.  CPU only."""
import os
from fractions import Fraction

import numpy as np

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
# fixture column -> stencil offset (di, dj, dk)
OFFS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def load():
    rows = []
    for line in open(os.path.join(HERE, "golden", "qs_eq17.txt")):
        if line.startswith("#") or not line.strip():
            continue
        left, right = line.split("|")
        d = [float(Fraction(t)) for t in left.split()]
        w = [float(Fraction(t)) for t in right.split()]
        rows.append((d, w))
    return rows


def test_qs_weights_match_eq17_golden_values():
    rows = load()
    assert len(rows) == 5
    for d, w in rows:
        offs, wt = O.shape_weights("qs", d)
        got = {tuple(int(x) for x in o): float(v) for o, v in zip(offs, wt)}
        assert set(got) == set(OFFS)
        for o, expect in zip(OFFS, w):
            assert abs(got[o] - expect) < 1e-15, (d, o, got[o], expect)
        assert abs(sum(w) - 1.0) < 1e-15
