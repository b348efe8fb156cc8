"""Writes bsf_knight_box_spline.h: the values of the grid box spline
beta'_b of the second direction set (boxes of one step along e1 = (2,1),
e2 = (1,2), e3 = (-1,2), e4 = (-2,1), unit mass), which interpolates that
set's running sums at continuous tap positions (Section 2.3, eq.
"interpolation", b = (sqrt 5, ...)), on the grid of 2^-6.

beta'_b(y) is the density of y = s1 e1 + s2 e2 + s3 e3 + s4 e4,
s ~ U[0,1]^4.  e1 is orthogonal to e3 (|e1 x e3| = 5), so with s = s2,
t = s4 and z = y - s e2 - t e4 the condition is 0 <= z.e1 <= 5,
0 <= z.e3 <= 5, i.e. for fixed s the admissible t form the interval
max(0, (4s - y.e1)/3, (y.e3 - 3s - 5)/4) <= t <= min(1, (5 + 4s - y.e1)/3,
(y.e3 - 3s)/4), and beta'_b(y) = (1/5) * integral over s in [0, 1] of its
length: a piecewise-linear function of s, integrated exactly between its
breakpoints (the crossings of the six bounds).

beta'_b is symmetric under the reflections of the square about its centre
(0, 3), so the table holds the fundamental domain: with (a, b) the centred
position in units of 2^-6, 0 <= b <= a <= 192,
kKnightBoxSpline[a (a + 1) / 2 + b] = beta'_b(a / 64, 3 + b / 64) * 491520,
an integer (491520 = 15 2^15; checked here for every entry).

Run: python gen_knight_box_spline.py  (writes the header beside this file).
"""
import os
from fractions import Fraction as Fr

DEN = 491520


def beta_kb(y1, y2):
    ye1 = 2 * y1 + y2
    ye3 = -y1 + 2 * y2
    # the bounds as (slope, intercept) in s
    lows = [(Fr(0), Fr(0)), (Fr(4, 3), -ye1 / 3), (Fr(-3, 4), (ye3 - 5) / 4)]
    highs = [(Fr(0), Fr(1)), (Fr(4, 3), (5 - ye1) / 3), (Fr(-3, 4), ye3 / 4)]
    lines = lows + highs
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
        lo = max(a * s + b for a, b in lows)
        hi = min(a * s + b for a, b in highs)
        return max(Fr(0), hi - lo)

    total = Fr(0)
    for a, b in zip(pts, pts[1:]):
        la, lb, lm = length(a), length(b), length((a + b) / 2)
        assert lm * 2 == la + lb  # linear on [a, b]: the trapezoid rule is exact
        total += (la + lb) / 2 * (b - a)
    return total / 5


def main():
    vals = []
    for a in range(193):
        for b in range(a + 1):
            v = beta_kb(Fr(a, 64), 3 + Fr(b, 64)) * DEN
            assert v.denominator == 1, (a, b, v)
            vals.append(int(v))
    assert sum(1 for v in vals if v < 0) == 0
    lines = ["// Generated by gen_knight_box_spline.py: the grid box spline beta'_b of the",
             "// second direction set on the grid of 2^-6 (see that script).  With (a, b)",
             "// the position relative to its centre (0, 3) in units of 2^-6, folded into",
             "// 0 <= b <= a <= 192 by the symmetries of the square, the value times",
             "// 491520 is kKnightBoxSpline[a (a + 1) / 2 + b].",
             "#pragma once", "",
             f"static __device__ const int kKnightBoxSpline[{len(vals)}] = {{"]
    for i in range(0, len(vals), 16):
        lines.append("    " + ", ".join(str(v) for v in vals[i:i + 16]) + ",")
    lines.append("};")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bsf_knight_box_spline.h")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(path, len(vals), max(vals))


if __name__ == "__main__":
    main()
