"""Writes qs_eq17.txt: the quadratic-sum deposit weights of Eq. 17 (App. B)
at a few rational relative coordinates, evaluated in exact rational
arithmetic straight from the printed formula (centre (3 - dx^2 - dy^2 -
dz^2)/6, face neighbours (1 +- d)^2/12).  It imports nothing of the
library or the oracle.

    python tests/golden/make_qs_eq17.py > tests/golden/qs_eq17.txt
"""
from fractions import Fraction as F

POINTS = [(F(0), F(0), F(0)), (F(1, 2), F(-1, 4), F(0)), (F(-3, 4), F(1, 3), F(7, 8)),
          (F(-1), F(1, 2), F(-1, 2)), (F(5, 16), F(-9, 16), F(3, 16))]

print("# Quadratic-sum deposit weights, Eq. 17 (App. B), exact rationals.")
print("# columns: dx dy dz | w(i,j,k) w(i+1) w(i-1) w(j+1) w(j-1) w(k+1) w(k-1)")
for dx, dy, dz in POINTS:
    w = [(3 - dx * dx - dy * dy - dz * dz) / 6,
         (1 + dx) ** 2 / 12, (1 - dx) ** 2 / 12,
         (1 + dy) ** 2 / 12, (1 - dy) ** 2 / 12,
         (1 + dz) ** 2 / 12, (1 - dz) ** 2 / 12]
    print(" ".join(str(v) for v in (dx, dy, dz)) + " | " + " ".join(str(v) for v in w))
