"""Writes bsf_grid_box_spline.h: the quadratic pieces of the grid box spline
beta_b (boxes of one step along d1 = (1,0), d2 = (1,1), d3 = (0,1),
d4 = (-1,1), unit mass) that interpolates the running sums at continuous tap
positions (Section 2.3, eq. "interpolation", read for the Cartesian set).

beta_b(y) is the density of y = s1 d1 + s2 d2 + s3 d3 + s4 d4, s ~ U[0,1]^4:
for fixed s = s2 the admissible t = s4 form the interval where
0 <= y1 - s + t <= 1, 0 <= y2 - s - t <= 1 and 0 <= t <= 1, so
beta_b(y) = integral over s in [0, 1] of its length, a piecewise-linear
function of s integrated exactly here between its breakpoints.  beta_b is
a quadratic on each triangle of the four-directional mesh (cells of the unit
grid cut by both diagonals); each piece is fitted through six exact values
and checked at ten more.

Pieces: cell (c1, c2), c1 in {-1, 0, 1}, c2 in {0, 1, 2}; triangle
0: v <= u, u + v <= 1; 1: v <= u, u + v >= 1; 2: v >= u, u + v >= 1;
3: v >= u, u + v <= 1 (u, v the position in the cell); six integers
k0..k5 with 8 beta_b(c + (u, v)) = k0 + k1 u + k2 v + k3 u^2 + k4 u v + k5 v^2,
written out as a device function of the integer position (U, V) = 1024 (u, v).

Run: python gen_grid_box_spline.py  (writes the header beside this file).
"""
import os
import random
from fractions import Fraction as Fr


def beta_b(y1, y2):
    lows = [lambda s: Fr(0), lambda s: s - y1, lambda s: y2 - s - 1]
    highs = [lambda s: Fr(1), lambda s: s - y1 + 1, lambda s: y2 - s]
    # breakpoints: where two bounds (each 0, 1, or +-s + const) cross; between
    # them the largest lower and the smallest upper bound are each one line,
    # and their difference changes sign only at such a crossing
    lines = [(0, Fr(0)), (0, Fr(1)), (1, -y1), (1, 1 - y1), (-1, y2), (-1, y2 - 1)]
    pts = {Fr(0), Fr(1)}
    for i in range(len(lines)):
        for j in range(i + 1, len(lines)):
            (a, b), (c, d) = lines[i], lines[j]
            if a != c:
                s = (d - b) / (a - c)
                if 0 < s < 1:
                    pts.add(s)
    pts = sorted(pts)

    def length(s):
        lo = max(f(s) for f in lows)
        hi = min(f(s) for f in highs)
        return max(Fr(0), hi - lo)

    total = Fr(0)
    for a, b in zip(pts, pts[1:]):
        la, lb, lm = length(a), length(b), length((a + b) / 2)
        assert lm * 2 == la + lb  # linear on [a, b]: the trapezoid rule is exact
        total += (la + lb) / 2 * (b - a)
    return total


def solve(A, b):
    n = len(A)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def inside(tri, u, v):
    return {0: v < u and u + v < 1, 1: v < u and u + v > 1, 2: v > u and u + v > 1, 3: v > u and u + v < 1}[tri]


def piece(c1, c2, tri, rng):
    pts = []
    while len(pts) < 16:
        u, v = Fr(rng.randrange(1, 97), 98), Fr(rng.randrange(1, 97), 98)
        if inside(tri, u, v) and (u, v) not in pts:
            pts.append((u, v))
    mono = lambda u, v: [Fr(1), u, v, u * u, u * v, v * v]  # noqa: E731
    a = solve([mono(u, v) for u, v in pts[:6]], [beta_b(c1 + u, c2 + v) for u, v in pts[:6]])
    for u, v in pts[6:]:
        assert sum(x * m for x, m in zip(a, mono(u, v))) == beta_b(c1 + u, c2 + v)
    k = [8 * x for x in a]
    assert all(x.denominator == 1 for x in k), k
    return [int(x) for x in k]


def main():
    rng = random.Random(0)
    rows = []
    for c1 in (-1, 0, 1):
        for c2 in (0, 1, 2):
            for tri in range(4):
                rows.append(((c1, c2, tri), piece(c1, c2, tri, rng)))
    # emitted as code: one branch per triangle, the nine weights with their
    # coefficients as constants.  The samples are loaded outside the branch:
    # the lanes of a warp rarely share the fractional tap position (the
    # steps carry nine fractional bits), and loads inside divergent branches
    # were measured to cost 30 % more than nine uniform loads.
    lines = ["// Generated by gen_grid_box_spline.py: the quadratic pieces of the grid box",
             "// spline beta_b (see that script).  For a tap at (floor, frac) = (z, (u, v)),",
             "// u = U / 1024, v = V / 1024, the weight of sample z + (i1, i2),",
             "// i1 in {-1, 0, 1}, i2 in {-2, -1, 0}, is beta_b(-i1 + u, -i2 + v) * 2^23 =",
             "// w[(i1 + 1) * 3 + (i2 + 2)] (cell c = (-i1, -i2)), with",
             "// 8 beta_b(c + (u, v)) = k0 + k1 u + k2 v + k3 u^2 + k4 u v + k5 v^2 per triangle",
             "// tri of the cell (0: v <= u, u + v <= 1; 1: v <= u, u + v >= 1;",
             "// 2: v >= u, u + v >= 1; 3: v >= u, u + v <= 1).",
             "#pragma once", "",
             "__device__ __forceinline__ void grid_box_spline_weights(int tri, int U, int V, int w[9]) {",
             "  const int UU = U * U, UV = U * V, VV = V * V;",
             "  switch (tri) {"]
    terms = ("(1 << 20)", "(U << 10)", "(V << 10)", "UU", "UV", "VV")
    for tri in range(4):
        lines.append(f"    {'default' if tri == 3 else 'case ' + str(tri)}:")
        for i1 in (-1, 0, 1):
            for i2 in (-2, -1, 0):
                c1, c2 = -i1, -i2
                k = dict(rows)[(c1, c2, tri)]
                expr = " + ".join(f"{v} * {t}" for v, t in zip(k, terms) if v) or "0"
                lines.append(f"      w[{(i1 + 1) * 3 + (i2 + 2)}] = {expr};  // cell ({c1}, {c2})")
        lines.append("      return;")
    lines += ["  }", "}"]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bsf_grid_box_spline.h")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(path)


if __name__ == "__main__":
    main()
