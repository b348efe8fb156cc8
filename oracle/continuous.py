"""Continuous-step filter (D2) and the derivative of its output with respect to
the covariance field.

Oracle module (test infrastructure only; see the package docstring).

Definition (the paper samples the running sums at off-grid points by
interpolation, Section 2.3, eq. "interpolation"; read here for the Cartesian
mesh with linear interpolation along each direction):

* The step lambda_k = sqrt(1 + A_k / |d_k|^2) of the minimum-kurtosis solve is
  not rounded to an integer.  It is quantised to 2^-(QW-1) of a grid step,
  H_k = RNE(2^(QW-1) lambda_k), lambda~ = H / 2^(QW-1), so that every
  interpolation fraction below is an exact multiple of 2^-QW (reading: a
  fixed-point step keeps the pipeline exact and keeps sum_t w_t q_t = 0, on
  which the compact support of the kernel rests).
* Along d_k the n-fold running sum is sampled at q_t = c - t lambda~,
  c = n (lambda~ - 1)/2, t = 0..n, by linear interpolation between the grid
  points a_t and a_t + 1 with q_t in [a_t, a_t + 1]:  a_t = floor(q_t) where
  q_t grows with lambda (t < n/2) and a_t = ceil(q_t) - 1 where it shrinks.
  (The two brackets agree on the value; they fix the one-sided derivative.)
  With theta_t = q_t - a_t in units of 2^-QW the sample weights are integers:
      v(a_t) += w_t (2^QW - theta_t),  v(a_t + 1) += w_t theta_t,
      w_t = (-1)^t C(n, t).
* The 1-D kernel of direction k is g(j) = sum_pos v(pos) P_n(pos - j), with
  P_n = C^n delta the n-fold running sum of an impulse (P_1(m) = [m >= 0],
  P_2(m) = (m + 1)[m >= 0]); the 2-D kernel is the convolution of the four
  1-D kernels placed on the lines Z d_k, and its mass M = prod_k M_k,
  M_k = sum_j g_k(j), normalises the output exactly like D1's prod L^n.
  For n = 2, g(j) = 2^QW max(0, lambda~ - |j|) (the triangle of half-width
  lambda~ sampled at the integers); for n = 1, g(j) = 2^QW times the overlap
  of [j - 1/2, j + 1/2) with [-lambda~/2, lambda~/2) (area sampling of the box).
  For n >= 3 the interpolated kernel has no compact support (the lerp does
  not reproduce quadratics), so the continuous path is defined for n <= 2.
  For lambda~ an admissible integer L the kernel is 2^QW times the D1 kernel
  of L in every direction.

Derivative (backward of the parameter fields): d out / d lambda_k takes the
derivative of the interpolation weights at the fixed brackets a_t,
dtheta_t / dlambda = n/2 - t, i.e. the right derivative of the continuous-step
filter at lambda~; the quantisation itself is passed through as the identity.
The chain to the covariance planes (or to log sigma, theta, log rho) is the
derivative of the float64 scale solve, taken here by complex-step
differentiation, so it shares no algebra with a hand-derived adjoint.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from functools import lru_cache
from math import comb

import numpy as np

from . import params
from .kernels import extend_image, extend_index
from .modular import U128, preintegrate
from .rounding import quantize, finalize

QW = 10
SCALE = 1 << QW          # interpolation weights are multiples of 2^-QW
HALF = SCALE // 2        # lambda is quantised to 2^-(QW-1)
H_MAX = HALF * params.L_MAX


def _check_order(n: int) -> None:
    if n not in (1, 2):
        raise ValueError("the continuous-step filter is defined for n = 1 and n = 2")


# ---------------------------------------------------------------------------
# steps
# ---------------------------------------------------------------------------

_F = np.float32
# Cody-Waite constants: ln 2 as a 16-bit head plus a tail, pi/2 as two 12-bit
# heads plus a tail (each head times a small integer is exact in float32)
LN2_HI, LN2_LO = _F(0.693145751953125), _F(1.428606765330187e-06)
LOG2E = _F(1.0 / math.log(2.0))
PIO2 = (_F(1.57080078125), _F(-4.453584551811218e-06), _F(-8.705516307827565e-10))
TWO_OVER_PI = _F(2.0 / math.pi)
INV_FACT = [_F(1.0 / math.factorial(k)) for k in range(11)]


def exp_f32(x):
    """e^x in float32 by Cody-Waite reduction x = k ln2 + r (|r| <= ln2/2) and
    the degree-7 Taylor polynomial of e^r, times 2^k; x clamped to [-87, 88].
    Every step is one IEEE float32 operation.  Pinned by tests: within 1.5
    ulp of float64 exp."""
    x = np.minimum(np.maximum(np.asarray(x, dtype=_F), _F(-87)), _F(88))
    kf = np.rint(x * LOG2E).astype(_F)
    r = ((x - kf * LN2_HI).astype(_F) - kf * LN2_LO).astype(_F)
    p = INV_FACT[7]
    for i in range(6, -1, -1):
        p = (p * r + INV_FACT[i]).astype(_F)
    scale = ((kf.astype(np.int32) + 127) << 23).astype(np.uint32).view(_F)
    return (p * scale).astype(_F)


def sincos_f32(x):
    """(sin x, cos x) in float32: Cody-Waite reduction x = j pi/2 + r
    (|r| <= pi/4, three-part pi/2), Taylor polynomials of degree 9 and 10 in
    r, the quadrant j mod 4 selecting and signing them.  Pinned by tests:
    within 2^-23 of float64 sin and cos on [-20, 20]."""
    x = np.asarray(x, dtype=_F)
    jf = np.rint(x * TWO_OVER_PI).astype(_F)
    r = x
    for part in PIO2:
        r = (r - jf * part).astype(_F)
    r2 = (r * r).astype(_F)
    c = INV_FACT
    sp = c[9]
    sp = (sp * r2 - c[7]).astype(_F)
    sp = (sp * r2 + c[5]).astype(_F)
    sp = (sp * r2 - c[3]).astype(_F)
    sp = ((sp * r2).astype(_F) * r + r).astype(_F)
    cp = -c[10]
    cp = (cp * r2 + c[8]).astype(_F)
    cp = (cp * r2 - c[6]).astype(_F)
    cp = (cp * r2 + c[4]).astype(_F)
    cp = (cp * r2 - c[2]).astype(_F)
    cp = (cp * r2 + _F(1)).astype(_F)
    j = jf.astype(np.int64) & 3
    sn = np.select([j == 0, j == 1, j == 2], [sp, cp, -sp], -cp).astype(_F)
    cs = np.select([j == 0, j == 1, j == 2], [cp, -sp, -cp], sp).astype(_F)
    return sn, cs


def cov_from_log_params(ls, th, lr):
    """(C11, C12, C22) as float32 from float32 planes (log sigma, theta, log rho).

    The covariance reading of the configs (trace 2 sigma^2, eigenvalue ratio
    rho, major axis at theta), evaluated in float32 with exp_f32 and
    sincos_f32, one IEEE operation per step in this order:
        s2 = exp(2 ls), rho = exp(lr), k = (2 s2) / (1 + rho),
        C11 = k (rho c^2 + s^2), C22 = k (rho s^2 + c^2),
        C12 = k ((rho - 1) (s c)).
    Pinned by tests against params.cov_from_sigma_rho_theta in float64.
    """
    ls = np.asarray(ls, dtype=_F)
    th = np.asarray(th, dtype=_F)
    lr = np.asarray(lr, dtype=_F)
    s2 = exp_f32((_F(2) * ls).astype(_F))
    rho = exp_f32(lr)
    k = ((_F(2) * s2).astype(_F) / (_F(1) + rho).astype(_F)).astype(_F)
    s, c = sincos_f32(th)
    cc = (c * c).astype(_F)
    ss = (s * s).astype(_F)
    sc = (s * c).astype(_F)
    c11 = (k * ((rho * cc).astype(_F) + ss).astype(_F)).astype(_F)
    c22 = (k * ((rho * ss).astype(_F) + cc).astype(_F)).astype(_F)
    c12 = (k * ((rho - _F(1)).astype(_F) * sc).astype(_F)).astype(_F)
    return c11, c12, c22


def covariance_planes(planes: np.ndarray, kind: int):
    """float32 (C11, C12, C22) of a [3][...] field of kind 0 (covariance) or 1
    (log sigma, theta, log rho)."""
    if kind == 0:
        return planes[0], planes[1], planes[2]
    if kind == 1:
        return cov_from_log_params(planes[0], planes[1], planes[2])
    raise ValueError(kind)


def half_steps(C11, C12, C22, n: int):
    """H_k = RNE(2^(QW-1) lambda_k) (int64 [4, ...]), lambda_k (float32) and flags.

    lambda_k comes from the float32 scale solve (params.solve_scales_f32) and
    the corrected step rule; the scaling by 2^(QW-1) is exact in float32."""
    _check_order(n)
    A, flags = params.solve_scales_f32(C11, C12, C22, n)
    lam = params.steps_from_scales(A, n, "corrected")
    Hs = np.rint(lam * np.float32(HALF)).astype(np.int64)
    return np.minimum(Hs, H_MAX), lam, flags


# ---------------------------------------------------------------------------
# one direction
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def line_taps(Hh: int, n: int):
    """Sample positions with integer weights and derivative weights.

    Returns (v, dv, dscale): dicts {position: weight} of the lerped samples,
    and of d v / d lambda times dscale (dscale = 2 for odd n, so that the
    derivative weights stay integers)."""
    _check_order(n)
    lam = 2 * Hh                  # lambda~ in units of 2^-QW
    c = n * (Hh - HALF)           # n (lambda~ - 1) / 2 in units of 2^-QW
    dscale = 2 if n % 2 else 1
    v, dv = {}, {}
    for t in range(n + 1):
        w = (-1) ** t * comb(n, t)
        Q = c - t * lam           # q_t in units of 2^-QW
        grows = n - 2 * t         # sign of d q_t / d lambda (times 2)
        a = Q // SCALE if grows >= 0 else -((-Q) // SCALE) - 1
        th = Q - a * SCALE
        assert 0 <= th <= SCALE
        v[a] = v.get(a, 0) + w * (SCALE - th)
        v[a + 1] = v.get(a + 1, 0) + w * th
        dq = grows * SCALE * dscale // 2      # (n/2 - t) 2^QW dscale
        dv[a] = dv.get(a, 0) - w * dq
        dv[a + 1] = dv.get(a + 1, 0) + w * dq
    return v, dv, dscale


def _P(n: int, m: int) -> int:
    """n-fold running sum of a unit impulse, evaluated at m."""
    if m < 0:
        return 0
    return 1 if n == 1 else m + 1


def line_kernel(weights: dict, n: int):
    """g(j) = sum_pos weights(pos) P_n(pos - j) on [min pos, max pos + 1].

    Returns (g as a tuple of ints, j0): g[i] is the weight at j = j0 + i.
    Raises if g does not vanish below its support (no compact support)."""
    lo, hi = min(weights), max(weights)
    val = lambda j: sum(w * _P(n, pos - j) for pos, w in weights.items())  # noqa: E731
    if val(lo - 1) != 0 or val(lo - 2) != 0:
        raise ArithmeticError("interpolated kernel without compact support")
    return tuple(val(j) for j in range(lo, hi + 2)), lo


def line_closed_form(Hh: int, n: int, j: int) -> int:
    """The 1-D kernel in closed form (2^QW times): triangle (n = 2) or box
    overlap (n = 1).  Used to pin line_kernel."""
    if n == 2:
        return max(0, 2 * Hh - SCALE * abs(j))
    if n == 1:
        return max(0, min(SCALE * j + HALF, Hh) - max(SCALE * j - HALF, -Hh))
    raise ValueError(n)


@lru_cache(maxsize=None)
def line_data(Hh: int, n: int):
    """(g, dg, j0, M, dM, dscale) of one direction: kernel, derivative kernel
    (times dscale) on a common index range starting at j0, and their sums."""
    v, dv, dscale = line_taps(Hh, n)
    g, j0 = line_kernel(v, n)
    dg, dj0 = line_kernel(dv, n) if any(dv.values()) else ((0,) * len(g), j0)
    lo = min(j0, dj0)
    hi = max(j0 + len(g), dj0 + len(dg))
    G = [0] * (hi - lo)
    D = [0] * (hi - lo)
    for i, x in enumerate(g):
        G[j0 - lo + i] += x
    for i, x in enumerate(dg):
        D[dj0 - lo + i] += x
    return tuple(G), tuple(D), lo, sum(G), sum(D), dscale


# ---------------------------------------------------------------------------
# 2-D kernels and the direct filter
# ---------------------------------------------------------------------------

def assemble(lines, dtype=object):
    """Convolution of four 1-D kernels [(g, j0)] placed on Z d_k (exact
    integers with dtype=object, float64 with dtype=np.float64).

    Returns (K, ox, oy): K[oy + dy, ox + dx] is the weight at offset (dx, dy)."""
    K = np.ones((1, 1), dtype=dtype)
    ox = oy = 0
    for k, (dx, dy) in enumerate(params.DIRS):
        g, j0 = lines[k]
        offs = np.arange(j0, j0 + len(g))
        sx, sy = offs * dx, offs * dy
        nx0, nx1 = -ox + sx.min(), K.shape[1] - 1 - ox + sx.max()
        ny0, ny1 = -oy + sy.min(), K.shape[0] - 1 - oy + sy.max()
        Kn = np.zeros((ny1 - ny0 + 1, nx1 - nx0 + 1), dtype=dtype)
        nox, noy = -nx0, -ny0
        for w, ddx, ddy in zip(g, sx, sy):
            if w == 0:
                continue
            y0 = noy - oy + ddy
            x0 = nox - ox + ddx
            Kn[y0:y0 + K.shape[0], x0:x0 + K.shape[1]] += w * K
        K, ox, oy = Kn, nox, noy
    return K, ox, oy


@lru_cache(maxsize=256)
def kernels_d2(Hs: tuple, n: int):
    """2-D kernel and its four derivative kernels for quantised steps Hs.

    Returns (K, dK[4], ox, oy, M, Mk[4], dMk[4], dscale); every kernel is laid
    out on the same (ox, oy) frame, dK[k] is K with direction k's 1-D kernel
    replaced by its derivative (times dscale)."""
    data = [line_data(int(h), n) for h in Hs]
    K, ox, oy = assemble([(d[0], d[2]) for d in data])
    dK = []
    for k in range(4):
        lines = [(d[0], d[2]) for d in data]
        lines[k] = (data[k][1], data[k][2])
        dk, dox, doy = assemble(lines)
        assert (dk.shape, dox, doy) == (K.shape, ox, oy)
        dK.append(dk)
    M = 1
    for d in data:
        M *= d[3]
    return K, dK, ox, oy, M, [d[3] for d in data], [d[4] for d in data], data[0][5]


def reach_d2(Hs, n: int) -> int:
    """Largest |offset| (x or y) of any sample of the continuous-step taps."""
    lo, hi = [], []
    for h in Hs:
        v, _, _ = line_taps(int(h), n)
        lo.append(min(v))
        hi.append(max(v))
    x_min = lo[0] + lo[1] - hi[3]
    x_max = hi[0] + hi[1] - lo[3]
    y_min = lo[1] + lo[2] + lo[3]
    y_max = hi[1] + hi[2] + hi[3]
    return max(-x_min, x_max, -y_min, y_max)


def _pixel_steps(planes, kind, n, y, x, R):
    C11, C12, C22 = covariance_planes(planes[:, y:y + 1, x:x + 1], kind)
    Hs, lam, flags = half_steps(C11, C12, C22, n)
    Hs = tuple(int(h) for h in Hs.reshape(4))
    far = R is not None and reach_d2(Hs, n) > R
    if far:  # out of reach: identity steps (the library flags it)
        Hs = (HALF,) * 4
    return Hs, lam.reshape(4), int(flags.reshape(())), far


def filter_d2_direct(fq: np.ndarray, planes: np.ndarray, n: int, boundary: int, pixels,
                     kind: int = 0, R: int | None = None):
    """Exact correlation sums of the definition at the given pixels.

    fq: integer image (int64 or object); planes: float32 [3][H][W] of the
    given kind.  Returns {(y, x): dict(acc, dacc[4], M, Mk[4], dMk[4], dscale,
    H[4], lam[4], far)} with exact Python integers."""
    H, W = fq.shape
    fobj = fq.astype(object)
    out = {}
    for (y, x) in pixels:
        Hs, lam, flags, far = _pixel_steps(planes, kind, n, y, x, R)
        K, dK, ox, oy, M, Mk, dMk, dscale = kernels_d2(Hs, n)
        kh, kw = K.shape
        yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
        xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
        patch = np.where(np.outer(yv, xv), fobj[np.ix_(yi, xi)], 0)
        out[(y, x)] = dict(acc=int((K * patch).sum()),
                           dacc=[int((d * patch).sum()) for d in dK],
                           M=M, Mk=Mk, dMk=dMk, dscale=dscale, H=Hs, lam=lam,
                           flags=flags, far=far)
    return out


# ---------------------------------------------------------------------------
# the paper's pipeline: running sums, then lerped taps
# ---------------------------------------------------------------------------

def _signed(v: int, bits: int) -> int:
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


def filter_d2_modular(f: np.ndarray, planes: np.ndarray, n: int, boundary: int, q: int,
                      bits: int = 128, kind: int = 0, R: int | None = None, pixels=None):
    """Running sums mod 2^bits (modular.preintegrate), then at each pixel the
    lerped taps: acc = sum over one sample position per direction of
    prod_k v_k(pos_k) S(p + sum_k pos_k d_k), and dacc_k with v_k -> dv_k.

    R defaults to the largest sample reach of the field (at least 3n);
    pixels defaults to every pixel.  Returns the same per-pixel dicts as
    filter_d2_direct, plus 'R'."""
    _check_order(n)
    Hh, Ww = f.shape
    C11, C12, C22 = covariance_planes(planes, kind)
    Hs_all, lam_all, flags_all = half_steps(C11, C12, C22, n)
    if pixels is None:
        pixels = [(y, x) for y in range(Hh) for x in range(Ww)]
    if R is None:
        R = 3 * n
        for y in range(Hh):
            for x in range(Ww):
                R = max(R, reach_d2(Hs_all[:, y, x], n))
    fq = quantize(f, q, as_object=(bits == 128))
    S = preintegrate(extend_image(fq, R, boundary), n, bits)
    if bits == 64:
        Sget = lambda yy, xx: int(S[yy, xx])  # noqa: E731
    else:
        Sget = lambda yy, xx: int(S.lo[yy, xx]) | (int(S.hi[yy, xx]) << 64)  # noqa: E731
    out = {}
    for (y, x) in pixels:
        Hs = tuple(int(h) for h in Hs_all[:, y, x])
        far = reach_d2(Hs, n) > R
        if far:
            Hs = (HALF,) * 4
        taps = [line_taps(h, n) for h in Hs]
        acc = 0
        dacc = [0, 0, 0, 0]
        lists = [sorted(t[0]) for t in taps]
        for combo in itertools.product(*lists):
            dxy = [0, 0]
            for k, pos in enumerate(combo):
                dxy[0] += pos * params.DIRS[k][0]
                dxy[1] += pos * params.DIRS[k][1]
            s = Sget(y + R + dxy[1], x + R + dxy[0])
            ws = [taps[k][0][pos] for k, pos in enumerate(combo)]
            dws = [taps[k][1].get(pos, 0) for k, pos in enumerate(combo)]
            prod = ws[0] * ws[1] * ws[2] * ws[3]
            acc += prod * s
            for k in range(4):
                if dws[k]:
                    other = 1
                    for j in range(4):
                        other *= dws[k] if j == k else ws[j]
                    dacc[k] += other * s
        datas = [line_data(h, n) for h in Hs]
        M = 1
        for d in datas:
            M *= d[3]
        out[(y, x)] = dict(acc=_signed(acc, bits), dacc=[_signed(a, bits) for a in dacc],
                           M=M, Mk=[d[3] for d in datas], dMk=[d[4] for d in datas],
                           dscale=datas[0][5], H=Hs, lam=lam_all[:, y, x],
                           flags=int(flags_all[y, x]), far=far, R=R)
    return out


# ---------------------------------------------------------------------------
# output and derivatives
# ---------------------------------------------------------------------------

def output(rec: dict, q: int, out_dtype=np.float32):
    """The output rule of rounding.finalize applied to one pixel's sums."""
    return finalize(np.array([rec["acc"]], dtype=object), np.array([rec["M"]], dtype=object),
                    q, out_dtype)[0]


def jacobian_steps(rec: dict, q: int):
    """d out / d lambda_k (float64, from the exact rational value):
    (dacc_k M_k - acc dM_k) / (dscale 2^q M M_k)."""
    out = []
    for k in range(4):
        num = rec["dacc"][k] * rec["Mk"][k] - rec["acc"] * rec["dMk"][k]
        den = rec["dscale"] * (1 << q) * rec["M"] * rec["Mk"][k]
        out.append(float(Fraction(num, den)))
    return np.array(out)


def solve_scales_f64(C11, C12, C22, n: int):
    """Minimum-kurtosis scales A_k in float64 for scalar inputs, complex-safe
    (comparisons on real parts), for complex-step differentiation.

    Same sanitising and clamping as solve_scales_f32; the stationarity cubic
    8u^3 - 6 s u^2 + (4(c1^2 + c3^2) + 8 b^2) u - (c1^3 + c3^3) - b^2 s = 0 is
    solved by Newton's method from its inflection point u = s/4 (monotone
    convergence), 80 steps.  Pinned by tests against solve_scales_bruteforce
    and by finite differences of its own real evaluation."""
    re = lambda z: z.real if isinstance(z, complex) else z  # noqa: E731
    c11 = C11 if re(C11) > 0 else 0.0 * C11
    c22 = C22 if re(C22) > 0 else 0.0 * C22
    m = c11 if re(c11) <= re(c22) else c22
    c12 = C12
    if abs(re(c12)) > re(m):
        c12 = m if re(c12) >= 0 else -m
    B = 12.0 / n
    c1, c3, b = B * c11, B * c22, B * c12
    s = c1 + c3
    u = s / 4.0
    for _ in range(80):
        g = 8 * u ** 3 - 6 * s * u ** 2 + (4 * (c1 * c1 + c3 * c3) + 8 * b * b) * u \
            - (c1 ** 3 + c3 ** 3) - b * b * s
        dg = 24 * u ** 2 - 12 * s * u + 4 * (c1 * c1 + c3 * c3) + 8 * b * b
        if re(dg) <= 0:
            break
        u = u - g / dg
    lo = b if re(b) >= 0 else -b
    hi = c1 if re(c1) <= re(c3) else c3
    if re(u) < re(lo):
        u = lo
    if re(u) > re(hi):
        u = hi
    return [c1 - u, u + b, c3 - u, u - b]


def steps_f64(p, kind: int, n: int):
    """Continuous steps lambda_k (float64, complex-safe) from one pixel's three
    planes of the given kind."""
    if kind == 0:
        C11, C12, C22 = p
    else:
        ls, th, lr = p
        s2 = np.exp(2.0 * ls)
        rho = np.exp(lr)
        k = (2.0 * s2) / (1.0 + rho)
        c, s = np.cos(th), np.sin(th)
        C11 = k * (rho * c * c + s * s)
        C22 = k * (rho * s * s + c * c)
        C12 = k * ((rho - 1.0) * s * c)
    A = solve_scales_f64(C11, C12, C22, n)
    return [np.sqrt(1.0 + A[k] / params.NORM2[k]) for k in range(4)]


def dsteps_dplanes(p, kind: int, n: int, h: float = 1e-30) -> np.ndarray:
    """[4][3] derivative of lambda_k with respect to the three planes, by
    complex-step differentiation of steps_f64 (no cancellation error)."""
    J = np.zeros((4, 3))
    for j in range(3):
        z = [complex(float(v)) for v in p]
        z[j] += complex(0.0, h)
        lam = steps_f64(z, kind, n)
        for k in range(4):
            J[k, j] = complex(lam[k]).imag / h
    return J


def jacobian_planes(rec: dict, p, kind: int, n: int, q: int) -> np.ndarray:
    """d out / d plane_j (3 values) at one pixel: chain of jacobian_steps and
    dsteps_dplanes.  Zero for a pixel outside the reach (identity steps)."""
    if rec["far"]:
        return np.zeros(3)
    return jacobian_steps(rec, q) @ dsteps_dplanes(p, kind, n)


# ---------------------------------------------------------------------------
# float64 continuous definition without quantisation (finite differences)
# ---------------------------------------------------------------------------

def line_kernel_real(lam: float, n: int):
    """The continuous-step 1-D kernel at a real lambda (no quantisation),
    normalised to unit mass: point samples of the triangle of half-width
    lambda (n = 2) or cell overlaps with the box of width lambda (n = 1)."""
    _check_order(n)
    r = int(math.ceil(lam)) + 1
    js = np.arange(-r, r + 1)
    if n == 2:
        g = np.maximum(0.0, lam - np.abs(js))
    else:
        g = np.maximum(0.0, np.minimum(js + 0.5, lam / 2) - np.maximum(js - 0.5, -lam / 2))
    return g / g.sum(), -r


def filter_d2_f64_at(f: np.ndarray, p, kind: int, n: int, boundary: int, y: int, x: int) -> float:
    """Continuous-step filter at one pixel with real (unquantised) steps from
    the float64 solve, in float64."""
    lams = [float(np.real(v)) for v in steps_f64([float(v) for v in p], kind, n)]
    K, ox, oy = assemble([line_kernel_real(l, n) for l in lams], dtype=np.float64)
    Hh, Ww = f.shape
    kh, kw = K.shape
    yi, yv = extend_index(np.arange(y - oy, y - oy + kh), Hh, boundary)
    xi, xv = extend_index(np.arange(x - ox, x - ox + kw), Ww, boundary)
    patch = np.where(np.outer(yv, xv), f[np.ix_(yi, xi)].astype(np.float64), 0.0)
    return math.fsum((K * patch).ravel().tolist())


def brackets(lam: float, n: int):
    """The interpolation brackets a_t at a real lambda (to detect kinks)."""
    c = n * (lam - 1.0) / 2.0
    out = []
    for t in range(n + 1):
        qt = c - t * lam
        out.append(math.floor(qt) if n - 2 * t >= 0 else math.ceil(qt) - 1)
    return tuple(out)


# ---------------------------------------------------------------------------
# adjoint with respect to the image
# ---------------------------------------------------------------------------

def grad_frac_bits_d2(max_abs_gout: float) -> int:
    """qg = 118 - ceil(log2 m) for m = max |gout| (float32), clamped to [0, 126]:
    the gradient sums are exact modulo 2^128 and keep 2^8 of headroom below
    2^127 (the rule of the integer-step backward, 54 = 62 - 8, moved to 128
    bits); 126 keeps 2^qg a float32."""
    m = float(np.float32(max_abs_gout))
    if m == 0.0 or not math.isfinite(m):
        c = 0
    else:
        mant, e = math.frexp(m)
        c = e - 1 if mant == 0.5 else e
    return int(min(max(118 - c, 0), 126))


def quantize_weight_d2(gout: float, M: int, qg: int) -> int:
    """g = RNE(RN32(RN32(gout 2^qg) / RN32(M))) as an exact Python integer."""
    from .rounding import rn_f32_int
    x = np.float32(np.float32(gout) * np.float32(math.ldexp(1.0, qg)))
    y = rn_f32_int(M)
    q = np.float32(x / y)
    return int(round(float(q)))  # round half to even; exact above 2^24


def adjoint_d2_acc(gq: dict, planes: np.ndarray, n: int, boundary: int, shape, kind: int = 0,
                   R: int | None = None):
    """Exact adjoint sums acc(x) = sum_p gq(p) K_p(x - p) folded onto the
    image by the extension rule, for integer weights gq {(y, x): int}.
    Python integers, object array [H][W]."""
    Hh, Ww = shape
    acc = np.zeros((Hh, Ww), dtype=object)
    for (y, x), g in gq.items():
        if g == 0:
            continue
        Hs, _, _, _ = _pixel_steps(planes, kind, n, y, x, R)
        K, _, ox, oy, *_ = kernels_d2(Hs, n)
        kh, kw = K.shape
        yi, yv = extend_index(np.arange(y - oy, y - oy + kh), Hh, boundary)
        xi, xv = extend_index(np.arange(x - ox, x - ox + kw), Ww, boundary)
        for a in range(kh):
            if not yv[a]:
                continue
            row = K[a] * g
            for b in range(kw):
                if xv[b] and row[b] != 0:
                    acc[yi[a], xi[b]] += row[b]
    return acc
