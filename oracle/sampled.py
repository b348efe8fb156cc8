"""The sampled continuous box spline: the filter the paper's interpolated
running sums compute (Section 2.3, eq. "interpolation"; Algorithm 3, step 3).

Oracle module (test infrastructure only; see the package docstring).

Reading.  With continuous scales the taps of the finite-difference mesh fall
between grid points, and the paper evaluates the running sum there by
interpolating its samples with the grid box spline beta_b of unit steps:
F(x) = sum_m g(m) beta_b(x - m).  The half-line running sum along d with unit
steps, convolved with the box of one step [0, d], is the continuous half-line
integral along d; so F is the continuous four-fold directional integral of
the image taken as point masses f(m) at the grid points, and the order-1
differences of F at the mesh's continuous offsets give

    out(p) = sum_m f(m) beta_a(p + tau - m),     tau = sum_k lambda_k d_k / 2,

the continuous box spline beta_a (boxes of lambda_k steps along d_k, unit
mass) sampled at the grid, centred.  This module computes that definition
directly and exactly (rational arithmetic), and also the paper's route
(running sums, interpolation by beta_b, differences) for small inputs; tests
pin the two equal.

beta_a with support sum_k [0, lambda_k d_k]: with (s, t) the positions along
d2 and d4 (in steps), x - s d2 - t d4 must lie in the rectangle
[0, lambda_1] x [0, lambda_3] spanned by d1 and d3, so

    beta_a(x) = area{(s, t) in [0, lambda_2] x [0, lambda_4] :
                     0 <= x1 - s + t <= lambda_1, 0 <= x2 - s - t <= lambda_3}
                / (lambda_1 lambda_2 lambda_3 lambda_4),

the area of a convex polygon (the rectangle in (s, t) clipped by four
half-planes), computed here by clipping and the shoelace formula in exact
fractions.  beta_b is the case lambda = (1, 1, 1, 1).

The second direction set (Algorithm 3 as printed: beta'_a interpolated by
beta'_b, eq. "interpolation" with b = (sqrt 5, ...)): boxes along
e1 = (2,1), e2 = (1,2), e3 = (-1,2), e4 = (-2,1); e1 is orthogonal to e3
and e2 to e4, so with z = x - s e2 - t e4 the condition is
z.e1 / 5 in [0, lambda_1], z.e3 / 5 in [0, lambda_3] (z.e1 = x.e1 - 4s + 3t,
z.e3 = x.e3 - 3s - 4t), and

    beta'_a(x) = area{(s, t) in [0, l2] x [0, l4] : ...} / (5 l1 l2 l3 l4),

the overlap of two rotated boxes the paper describes for beta'_b.  Steps
lambda_k = a_k / sqrt(5) quantised to 5 fractional bits (Lq = max(1,
RNE(32 lambda))), so the taps lie on the grid of 2^-6, where the values of
beta'_b times 491520 = 15 2^15 are integers; out = RN(RN(acc) 2^(5 - q)) /
RN(15 prod Lq).

Steps of beta_a: n = 1 (the paper's order).  lambda_k = a_k / |d_k| from the
minimum-kurtosis scales (the continuous box spline has covariance
sum_k a_k^2 u_k u_k^T / 12 = C exactly, so no step correction), computed in
float32 as sqrt(A_k / |d_k|^2) and quantised to K = 9 fractional bits:
Lq_k = max(1, RNE(512 lambda_k)), lambda_k = Lq_k / 512.  Every tap then sits
on the grid of 2^-10, beta_b's pieces are quadratics on the four-directional
mesh, and the interpolation weights are integers over 2^23.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import params
from .kernels import extend_index
from .rounding import quantize, rn_f32_int, rn_f64_int

K_BITS = 9
SCALE = 1 << K_BITS          # lambda = Lq / 512
WEIGHT_BITS = 2 * K_BITS + 5  # beta_b values are integers over 2^23 at taps on the 2^-10 grid

_F = np.float32


def lambdas_q(C11, C12, C22):
    """Quantised steps Lq[4] (int64) and flags from the covariance (n = 1).

    lambda_k = sqrt(A_k / |d_k|^2) in float32 (A from params.solve_scales_f32),
    Lq = max(1, RNE(512 lambda)) (512 lambda is exact in float32)."""
    A, flags = params.solve_scales_f32(C11, C12, C22, 1)
    A = np.asarray(A, dtype=_F)
    nrm = np.array([_F(1), _F(0.5), _F(1), _F(0.5)], dtype=_F).reshape((4,) + (1,) * (A.ndim - 1))
    lam = np.sqrt((A * nrm).astype(_F)).astype(_F)
    Lq = np.rint((lam * _F(SCALE)).astype(_F)).astype(np.int64)
    return np.maximum(Lq, 1), flags


# --------------------------------------------------------------------------
# Exact polygon areas
# --------------------------------------------------------------------------

def _clip(poly, a, b, c):
    """Keep the part of the polygon with a*s + b*t <= c (Sutherland-Hodgman)."""
    out = []
    n = len(poly)
    for i in range(n):
        P, Q = poly[i], poly[(i + 1) % n]
        fp = a * P[0] + b * P[1] - c
        fq = a * Q[0] + b * Q[1] - c
        if fp <= 0:
            out.append(P)
        if (fp < 0 < fq) or (fq < 0 < fp):
            r = fp / (fp - fq)
            out.append((P[0] + r * (Q[0] - P[0]), P[1] + r * (Q[1] - P[1])))
    return out


def _area(poly):
    n = len(poly)
    if n < 3:
        return Fraction(0)
    s = Fraction(0)
    for i in range(n):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % n]
        s += x0 * y1 - x1 * y0
    return abs(s) / 2


def overlap_area(x1, x2, lam):
    """area{(s, t) in [0, l2] x [0, l4] : 0 <= x1 - s + t <= l1, 0 <= x2 - s - t <= l3}
    (Fractions in, Fraction out)."""
    l1, l2, l3, l4 = lam
    poly = [(Fraction(0), Fraction(0)), (l2, Fraction(0)), (l2, l4), (Fraction(0), l4)]
    for a, b, c in ((1, -1, x1), (-1, 1, l1 - x1), (1, 1, x2), (-1, -1, l3 - x2)):
        # s - t <= x1;  t - s <= l1 - x1;  s + t <= x2;  -(s + t) <= l3 - x2
        poly = _clip(poly, a, b, Fraction(c))
        if not poly:
            return Fraction(0)
    return _area(poly)


def beta(x1, x2, lam):
    """beta_a(x) with support sum_k [0, lambda_k d_k] (exact)."""
    l1, l2, l3, l4 = lam
    return overlap_area(x1, x2, lam) / (l1 * l2 * l3 * l4)


def lam_of(Lq):
    return tuple(Fraction(int(v), SCALE) for v in Lq)


# --------------------------------------------------------------------------
# The definition: out(p) = sum_m f(m) beta_a(p + tau - m)
# --------------------------------------------------------------------------

def exact_value(fq, Lq, boundary, y, x):
    """sum_m Q(m) beta_a(p + tau - m) as a Fraction, p = (x, y), Q the
    quantised image extended by the boundary rule."""
    H, W = fq.shape
    lam = lam_of(Lq)
    tx = (lam[0] + lam[1] - lam[3]) / 2
    ty = (lam[1] + lam[2] + lam[3]) / 2
    cx, cy = Fraction(x) + tx, Fraction(y) + ty
    # support of beta_a: x in [-l4, l1 + l2], y in [0, l2 + l3 + l4]
    mx0 = math.floor(cx - lam[0] - lam[1])
    mx1 = math.ceil(cx + lam[3])
    my0 = math.floor(cy - lam[1] - lam[2] - lam[3])
    my1 = math.ceil(cy)
    ys, yv = extend_index(np.arange(my0, my1 + 1), H, boundary)
    xs, xv = extend_index(np.arange(mx0, mx1 + 1), W, boundary)
    acc = Fraction(0)
    for iy, m2 in enumerate(range(my0, my1 + 1)):
        if not yv[iy]:
            continue
        for ix, m1 in enumerate(range(mx0, mx1 + 1)):
            if not xv[ix]:
                continue
            v = int(fq[ys[iy], xs[ix]])
            if v:
                acc += v * beta(cx - m1, cy - m2, lam)
    return acc


def accumulator(value, Lq):
    """The integer accumulator of the running-sum route: value * prod(512 lambda)
    / 2^(4K - 23); exact (asserts integrality)."""
    prodL = 1
    for v in Lq:
        prodL *= int(v)
    a = value * prodL * Fraction(1 << WEIGHT_BITS, 1 << (4 * K_BITS))
    assert a.denominator == 1, a
    return a.numerator


def output(acc: int, Lq, q: int, out_dtype=np.float32):
    """out = RN(RN(acc) 2^(4K - 23 - q)) / RN(prod Lq) (float32 or float64)."""
    prodL = 1
    for v in Lq:
        prodL *= int(v)
    e = 4 * K_BITS - WEIGHT_BITS - q
    if np.dtype(out_dtype) == np.float32:
        a = rn_f32_int(acc)
        return np.float32(np.float32(a * np.float32(math.ldexp(1.0, e))) / rn_f32_int(prodL))
    a = rn_f64_int(acc)
    return np.float64((a * math.ldexp(1.0, e)) / rn_f64_int(prodL))


def filter_sampled(f, cov, boundary, q, out_dtype=np.float32, pixels=None):
    """Forward filter by the definition; all pixels, or a dict for `pixels`."""
    H, W = f.shape
    fq = quantize(f, q, as_object=True)
    Lq, flags = lambdas_q(cov[0], cov[1], cov[2])
    it = pixels if pixels is not None else [(y, x) for y in range(H) for x in range(W)]
    res = {}
    for (y, x) in it:
        L = Lq[:, y, x]
        res[(y, x)] = output(accumulator(exact_value(fq, L, boundary, y, x), L), L, q, out_dtype)
    if pixels is not None:
        return res
    out = np.empty((H, W), dtype=out_dtype)
    for (y, x), v in res.items():
        out[y, x] = v
    return out


def reach(Lq):
    """Padding R the running-sum route needs: the taps lie within
    sum_k lambda_k |d_k|_inf / 2 of the pixel, and the interpolation reaches
    one sample left, right and up, two down (rounded up)."""
    Lq = np.asarray(Lq, dtype=np.int64)
    half = (Lq[0] + Lq[1] + Lq[3] + SCALE - 1) // SCALE, (Lq[1] + Lq[2] + Lq[3] + SCALE - 1) // SCALE
    return np.maximum(half[0], half[1]) // 2 + 3


# --------------------------------------------------------------------------
# The paper's route, for pinning: running sums, interpolation, differences
# --------------------------------------------------------------------------

def paper_route_value(fq, Lq, boundary, y, x, R):
    """(1/prod lambda) sum_t (-1)^|t| F(p + sum_k (1/2 - t_k) lambda_k d_k), with
    F(z) = sum_m g(m) beta_b(z - m) and g the four running sums of the
    extended image on the padded domain [-R, W+R) x [-R, H+R) (Python ints,
    no modulus).  Returns a Fraction."""
    import itertools
    H, W = fq.shape
    Hp, Wp = H + 2 * R, W + 2 * R
    yi, yv = extend_index(np.arange(-R, H + R), H, boundary)
    xi, xv = extend_index(np.arange(-R, W + R), W, boundary)
    g = [[int(fq[yi[a], xi[b]]) if (yv[a] and xv[b]) else 0 for b in range(Wp)] for a in range(Hp)]
    for dx, dy in ((1, 0), (0, 1), (1, 1), (-1, 1)):
        for a in range(Hp):
            for b in range(Wp):
                pa, pb = a - dy, b - dx
                if 0 <= pa < Hp and 0 <= pb < Wp:
                    g[a][b] += g[pa][pb]
    lam = lam_of(Lq)
    ones = (Fraction(1),) * 4
    total = Fraction(0)
    for t in itertools.product((0, 1), repeat=4):
        zx, zy = Fraction(x), Fraction(y)
        for k, (dx, dy) in enumerate(((1, 0), (1, 1), (0, 1), (-1, 1))):
            c = (Fraction(1, 2) - t[k]) * lam[k]
            zx += c * dx
            zy += c * dy
        F = Fraction(0)
        for m2 in range(math.floor(zy) - 3, math.floor(zy) + 1):
            for m1 in range(math.floor(zx) - 2, math.floor(zx) + 2):
                w = beta(zx - m1, zy - m2, ones)
                if w:
                    F += g[m2 + R][m1 + R] * w
        total += (-1) ** sum(t) * F
    return total / (lam[0] * lam[1] * lam[2] * lam[3])


# --------------------------------------------------------------------------
# The second direction set: beta'_a, beta'_b
# --------------------------------------------------------------------------

K_BITS_K = 5
SCALE_K = 1 << K_BITS_K       # lambda = Lq / 32
WEIGHT_DEN_K = 491520         # beta'_b * 15 * 2^15 is an integer on the 2^-6 grid


def lambdas_q_k(C11, C12, C22):
    """Quantised steps of beta'_a: lambda_k = sqrt(3A_k / 15) in float32 (3A
    from knight.solve_scales_k_f32, n = 1), Lq = max(1, RNE(32 lambda))."""
    from . import knight
    A3, flags = knight.solve_scales_k_f32(C11, C12, C22, 1)
    lam = knight.steps_from_scales_k(A3, 1, "paper")
    Lq = np.rint((lam * _F(SCALE_K)).astype(_F)).astype(np.int64)
    return np.maximum(Lq, 1), flags


def overlap_area_k(x1, x2, lam):
    """area{(s, t) in [0, l2] x [0, l4] : 0 <= x.e1 - 4s + 3t <= 5 l1,
    0 <= x.e3 - 3s - 4t <= 5 l3} (Fractions)."""
    l1, l2, l3, l4 = lam
    xe1 = 2 * x1 + x2
    xe3 = -x1 + 2 * x2
    poly = [(Fraction(0), Fraction(0)), (l2, Fraction(0)), (l2, l4), (Fraction(0), l4)]
    for a, b, c in ((4, -3, xe1), (-4, 3, 5 * l1 - xe1), (3, 4, xe3), (-3, -4, 5 * l3 - xe3)):
        poly = _clip(poly, a, b, Fraction(c))
        if not poly:
            return Fraction(0)
    return _area(poly)


def beta_k(x1, x2, lam):
    """beta'_a(x), support sum_k [0, lambda_k e_k] (exact)."""
    l1, l2, l3, l4 = lam
    return overlap_area_k(x1, x2, lam) / (5 * l1 * l2 * l3 * l4)


def lam_of_k(Lq):
    return tuple(Fraction(int(v), SCALE_K) for v in Lq)


_E = ((2, 1), (1, 2), (-1, 2), (-2, 1))


def exact_value_k(fq, Lq, boundary, y, x):
    """sum_m Q(m) beta'_a(p + tau - m) as a Fraction, tau = sum_k lambda_k e_k / 2."""
    H, W = fq.shape
    lam = lam_of_k(Lq)
    tx = sum(l * e[0] for l, e in zip(lam, _E)) / 2
    ty = sum(l * e[1] for l, e in zip(lam, _E)) / 2
    cx, cy = Fraction(x) + tx, Fraction(y) + ty
    # support of beta'_a: x in [-(l3 + 2 l4), 2 l1 + l2], y in [0, l1 + 2 l2 + 2 l3 + l4]
    mx0 = math.floor(cx - 2 * lam[0] - lam[1])
    mx1 = math.ceil(cx + lam[2] + 2 * lam[3])
    my0 = math.floor(cy - lam[0] - 2 * lam[1] - 2 * lam[2] - lam[3])
    my1 = math.ceil(cy)
    ys, yv = extend_index(np.arange(my0, my1 + 1), H, boundary)
    xs, xv = extend_index(np.arange(mx0, mx1 + 1), W, boundary)
    acc = Fraction(0)
    for iy, m2 in enumerate(range(my0, my1 + 1)):
        if not yv[iy]:
            continue
        for ix, m1 in enumerate(range(mx0, mx1 + 1)):
            if not xv[ix]:
                continue
            v = int(fq[ys[iy], xs[ix]])
            if v:
                acc += v * beta_k(cx - m1, cy - m2, lam)
    return acc


def accumulator_k(value, Lq):
    """value * prod(32 lambda) * 491520 / 32^4: the integer accumulator of the
    running-sum route (asserts integrality)."""
    prodL = 1
    for v in Lq:
        prodL *= int(v)
    a = value * prodL * Fraction(WEIGHT_DEN_K, SCALE_K ** 4)
    assert a.denominator == 1, a
    return a.numerator


def output_k(acc: int, Lq, q: int, out_dtype=np.float32):
    """out = RN(RN(acc) 2^(5 - q)) / RN(15 prod Lq)."""
    M = 15
    for v in Lq:
        M *= int(v)
    e = 4 * K_BITS_K - 15 - q
    if np.dtype(out_dtype) == np.float32:
        a = rn_f32_int(acc)
        return np.float32(np.float32(a * np.float32(math.ldexp(1.0, e))) / rn_f32_int(M))
    a = rn_f64_int(acc)
    return np.float64((a * math.ldexp(1.0, e)) / rn_f64_int(M))


def reach_k(Lq):
    """Padding the second set's sampled taps need: the taps within
    (2 l1 + l2 + l3 + 2 l4)/2 across and (l1 + 2 l2 + 2 l3 + l4)/2 down of the
    pixel, the interpolation three samples around (rounded up)."""
    Lq = np.asarray(Lq, dtype=np.int64)
    sx = 2 * Lq[0] + Lq[1] + Lq[2] + 2 * Lq[3]
    sy = Lq[0] + 2 * Lq[1] + 2 * Lq[2] + Lq[3]
    cx = (sx + SCALE_K - 1) // SCALE_K
    cy = (sy + SCALE_K - 1) // SCALE_K
    return np.maximum(cx, cy) // 2 + 7


def filter_sampled_k(f, cov, boundary, q, out_dtype=np.float32, pixels=None):
    """The second set's sampled box spline by the definition."""
    H, W = f.shape
    fq = quantize(f, q, as_object=True)
    Lq, _ = lambdas_q_k(cov[0], cov[1], cov[2])
    it = pixels if pixels is not None else [(y, x) for y in range(H) for x in range(W)]
    res = {}
    for (y, x) in it:
        L = Lq[:, y, x]
        res[(y, x)] = output_k(accumulator_k(exact_value_k(fq, L, boundary, y, x), L), L, q, out_dtype)
    if pixels is not None:
        return res
    out = np.empty((H, W), dtype=out_dtype)
    for (y, x), v in res.items():
        out[y, x] = v
    return out


def filter_sampled_pair(f, cov, boundary, q, out_dtype=np.float32, pixels=None):
    """Algorithm 2 with the sampled box splines: per pixel beta_a or beta'_a by
    the sector of knight.use_knight."""
    from . import knight
    H, W = f.shape
    mask = knight.use_knight(cov[0], cov[1], cov[2])
    it = pixels if pixels is not None else [(y, x) for y in range(H) for x in range(W)]
    a = filter_sampled(f, cov, boundary, q, out_dtype, pixels=[p for p in it if not mask[p]])
    b = filter_sampled_k(f, cov, boundary, q, out_dtype, pixels=[p for p in it if mask[p]])
    a.update(b)
    if pixels is not None:
        return a
    out = np.empty((H, W), dtype=out_dtype)
    for (y, x), v in a.items():
        out[y, x] = v
    return out


def paper_route_value_k(fq, Lq, boundary, y, x, R):
    """Algorithm 3 as printed, in exact arithmetic: the running sums along
    e1..e4 (Python ints), interpolated at the 16 taps by beta'_b (support
    within [-3, 3] x [0, 6] of the sample), differenced, over prod lambda."""
    import itertools
    H, W = fq.shape
    Hp, Wp = H + 2 * R, W + 2 * R
    yi, yv = extend_index(np.arange(-R, H + R), H, boundary)
    xi, xv = extend_index(np.arange(-R, W + R), W, boundary)
    g = [[int(fq[yi[a], xi[b]]) if (yv[a] and xv[b]) else 0 for b in range(Wp)] for a in range(Hp)]
    for dx, dy in _E:
        for a in range(Hp):
            for b in range(Wp):
                pa, pb = a - dy, b - dx
                if 0 <= pa < Hp and 0 <= pb < Wp:
                    g[a][b] += g[pa][pb]
    lam = lam_of_k(Lq)
    ones = (Fraction(1),) * 4
    total = Fraction(0)
    for t in itertools.product((0, 1), repeat=4):
        zx, zy = Fraction(x), Fraction(y)
        for k, (dx, dy) in enumerate(_E):
            c = (Fraction(1, 2) - t[k]) * lam[k]
            zx += c * dx
            zy += c * dy
        F = Fraction(0)
        for m2 in range(math.floor(zy) - 6, math.floor(zy) + 1):
            for m1 in range(math.floor(zx) - 3, math.floor(zx) + 4):
                w = beta_k(zx - m1, zy - m2, ones)
                if w:
                    F += g[m2 + R][m1 + R] * w
        total += (-1) ** sum(t) * F
    return total / (lam[0] * lam[1] * lam[2] * lam[3])
