"""Writes axial_tangency.txt: exact Apollonius tangency cases of an axial wire (tan tau = 0).

Section 2.1 of the paper: for an axial wire the drift circle (centre = wire, radius = d) is
tangent to the helix's base circle, |W - C| = R + d (external) or |W - C| = R - d
(internal); Eq. (ApoEQ3D) with tan tau = 0 reduces to F = |W - C|^2 - (R +- d)^2.
Every coordinate below is dyadic, so F, and rho F with rho = 1/R a power of two, are exact
binary fractions: the interval program must return them as thin, exact intervals.

The expected values come from this closed form in exact rational arithmetic (fractions),
not from any implementation of the method.
"""
from fractions import Fraction as Fr
import itertools
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    rows = []
    phis = [(Fr(0), Fr(1)), (Fr(1), Fr(0)), (Fr(0), Fr(-1)), (Fr(-1), Fr(0))]  # (sin, cos) of phi0
    dirs = [(3, 4, 5), (-4, 3, 5), (5, -12, 13), (-8, -15, 17)]
    for R, (s0, c0), d0, (a, b, c), scale in itertools.product(
            [Fr(1), Fr(2), Fr(4)], phis, [Fr(0), Fr(1, 4), Fr(-1, 8)], dirs,
            [Fr(1, 4), Fr(1, 16)]):
        xc, yc = -(R + d0) * s0, (R + d0) * c0            # centre, Eq. (HelixEq_d)
        x0, y0 = xc + a * scale, yc + b * scale           # |W - C| = c * scale
        dist = c * scale
        cases = []
        if dist > R:
            cases.append(dist - R)        # external tangency: |W - C| = R + d
        if dist < R:
            cases.append(R - dist)        # internal tangency: |W - C| = R - d
        cases.append(Fr(3, 32))           # generic drift: no tangency unless by chance
        for d in cases:
            A2 = dist * dist
            gp = (A2 - (R + d) ** 2) / R
            gm = (A2 - (R - d) ** 2) / R
            vote = int(gp == 0 or gm == 0)
            rows.append((s0, c0, 1 / R, d0, x0, y0, d, gp, gm, vote))
    path = os.path.join(HERE, "axial_tangency.txt")
    with open(path, "w") as f:
        f.write("# Exact axial Apollonius tangency (paper Section 2.1; Eq. ApoEQ3D with tan tau = 0)\n")
        f.write("# columns: sin_phi0 cos_phi0 omega d0 x0 y0 drift G+ G- vote ; G = rho * F, rationals p/q\n")
        f.write("# written by make_axial_tangency.py from the closed form |W-C|^2 - (R +- d)^2\n")
        for r in rows:
            f.write(" ".join(str(v) for v in r) + "\n")
    print(path, len(rows))


if __name__ == "__main__":
    main()
