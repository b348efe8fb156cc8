"""The second four-directional box spline beta'_a and the pair of box splines
(Section 2.3: Algorithms 2 and 3, Table 1).

Oracle module (test infrastructure only; see the package docstring).

Directions.  beta'_a places its boxes along the near-uniform rational
directions of Section 2.3, tan = 1/2, 2, -2, -1/2 (26.6, 63.4, 116.6 and
153.4 degrees).  As grid vectors (x the column, y the row), matching the
mesh of Table 1 (tap 1 at a'_1 (2, 1), tap 2 at a'_2 (1, 2), tap 4 at
a'_3 (-1, 2), tap 8 at a'_4 (-2, 1)):

    e_1 = (2, 1), e_2 = (1, 2), e_3 = (-1, 2), e_4 = (-2, 1),  |e_k|^2 = 5.

Covariance (Section 2.3): C = (1/60) [[4A1 + A2 + A3 + 4A4, 2(A1 + A2 - A3 - A4)],
[., A1 + 4A2 + 4A3 + A4]] = (1/12) sum_k A_k u_k u_k^T, A_k = a_k^2,
u_k = e_k / sqrt(5); n times that for the n-fold filter.

Scale family (derivation, not printed in the paper).  With M = (12/n) C the
three equations fix P = A1 + A4 = (4 M11 - M22)/3, Q = A2 + A3 =
(4 M22 - M11)/3 and A1 + A2 - A3 - A4 = m, m = (5/2) M12; the null direction
is (1, -1, 1, -1), so with t = A1:
    A1 = t, A2 = (P + Q + m)/2 - t, A3 = (Q - P - m)/2 + t, A4 = P - t,
feasible (all A_k >= 0) for max(0, (P - Q + m)/2) <= t <= min(P, (P + Q + m)/2),
which is non-empty iff P >= 0, Q >= 0 and |m| <= P + Q, i.e.
    4 C11 >= C22,  4 C22 >= C11,  |C12| <= (2/5)(C11 + C22).
This is the elongation bound of beta'_a, elongation_bound_k below; the paper
found it by search (Table 4, "new bound" row).

Minimum kurtosis (Section 2.3): the paper prints the kurtosis matrix
(kappa/5) [[4a1^4 + a2^4 + a3^4 + 4a4^4, 2(a1^4 + a2^4 - a3^4 - a4^4)], [.,
a1^4 + 4a2^4 + 4a3^4 + a4^4]] = kappa sum_k A_k^2 u_k u_k^T and minimises its
Frobenius norm F.  Along the family dF/dt = 0 is a cubic; with
t = P/2 + m/4 + v it is depressed,
    v^3 + p v + q = 0,  p = (82 P^2 - 64 P Q + 82 Q^2 + 43 m^2)/400,
                        q = m (P^2 - Q^2)/32,
p > 0, so the cubic is strictly increasing (F is convex along the family).

Pair of box splines (Algorithm 2).  Each pixel uses beta'_a where its
orientation lies in the sector S' where beta'_a reaches the larger
elongation (Table 4: "the new bound is the maximum of the bounds of the two
box splines"), else beta_a.  Folding the orientation into [0, 45] degrees
(both bounds share the symmetries of the square) and writing t = tan(phi),
the two bounds in the form (e + 1)/(e - 1) are
    beta:   (1 + 2t - t^2)/(1 + t^2),
    beta':  max((5/3)(1 - t^2), (5/2) t)/(1 + t^2),
so beta' is the larger bound iff t^2 + 3t - 1 > 0 and 2t^2 + t - 2 < 0
(16.85 < phi < 37.98 degrees), which in terms of C, with t = tan(psi/2) and
(cos psi, sin psi) proportional to (|C11 - C22|, 2|C12|), reads
    |C11 - C22| < 3 |C12|  and  |C12| < 2 |C11 - C22|.
"""
from __future__ import annotations

import itertools
import math
from math import comb

import numpy as np

from . import params
from .kernels import correlate_exact, extend_image, kernel_mass
from .modular import U128, U64, MASK64
from .rounding import finalize, quantize

DIRS_K = ((2, 1), (1, 2), (-1, 2), (-2, 1))
NORM2_K = 5

_F = np.float32


# --------------------------------------------------------------------------
# Geometry of beta'_a
# --------------------------------------------------------------------------

def covariance_of_scales_k(a, n: int = 1) -> np.ndarray:
    """Covariance of the n-fold beta'_a (the paper's (1/60) matrix, times n)."""
    q = np.asarray(a, dtype=np.float64) ** 2
    c11 = 4 * q[0] + q[1] + q[2] + 4 * q[3]
    c12 = 2 * (q[0] + q[1] - q[2] - q[3])
    c22 = q[0] + 4 * q[1] + 4 * q[2] + q[3]
    return (n / 60.0) * np.array([[c11, c12], [c12, c22]])


def geometry_of_scales_k(a):
    """(size r/60, elongation, orientation) of beta'_a from the paper's p, q, r:
    p = 3(A1 - A2 - A3 + A4), q = 4(A1 + A2 - A3 - A4), r = 5 sum A,
    elongation (r + sqrt(p^2 + q^2))/(r - sqrt(p^2 + q^2)),
    tan(orientation) = (-p + sqrt(p^2 + q^2))/q."""
    A = np.asarray(a, dtype=np.float64) ** 2
    p = 3 * (A[0] - A[1] - A[2] + A[3])
    q = 4 * (A[0] + A[1] - A[2] - A[3])
    r = 5 * A.sum()
    s = math.hypot(p, q)
    rho = (r + s) / (r - s) if r > s else math.inf
    if q == 0.0:
        theta = 0.0 if p >= 0 else math.pi / 2
    else:
        theta = math.atan((-p + s) / q) % math.pi
    return r / 60.0, rho, theta


def kurtosis_matrix_k(A) -> np.ndarray:
    """sum_k A_k^2 u_k u_k^T (the paper's matrix without the factor kappa)."""
    A = np.asarray(A, dtype=np.float64)
    M = np.zeros((2, 2))
    for k, (ex, ey) in enumerate(DIRS_K):
        u = np.array([ex, ey], dtype=np.float64) / math.sqrt(NORM2_K)
        M += A[k] ** 2 * np.outer(u, u)
    return M


def kurtosis_objective_k(A) -> float:
    M = kurtosis_matrix_k(A)
    return float((M * M).sum())


def feasible_k(C11, C12, C22) -> bool:
    """True when some A >= 0 has covariance C (the beta'_a elongation bound)."""
    return 4 * C11 >= C22 and 4 * C22 >= C11 and abs(C12) <= 0.4 * (C11 + C22)


def elongation_bound_k(phi) -> float:
    """Largest elongation beta'_a reaches at orientation phi (closed form of
    feasible_k for C = R(phi) diag(e, 1) R(phi)^T, folded into [0, 45] degrees)."""
    phi = float(phi) % math.pi
    phi = min(phi, math.pi - phi)          # reflection about the x axis
    phi = min(phi, math.pi / 2 - phi) if phi <= math.pi / 2 else phi
    t = math.tan(phi)
    ratios = []
    if t < 0.5:
        ratios.append((5.0 / 3.0) * (1 - t * t) / (1 + t * t))   # 4 C22 >= C11
    if t > 0.5:
        ratios.append(2.5 * t / (1 + t * t))                     # |C12| <= 0.4 (C11 + C22)
    if not ratios:
        return math.inf
    r = max(ratios)
    return math.inf if r <= 1.0 else (r + 1.0) / (r - 1.0)


def scale_family_k(C11, C12, C22, n: int, t):
    """A(t) of the one-parameter family with covariance C (float64)."""
    B = 12.0 / n
    M11, M12, M22 = B * C11, B * C12, B * C22
    P = (4 * M11 - M22) / 3.0
    Q = (4 * M22 - M11) / 3.0
    m = 2.5 * M12
    return np.array([t, (P + Q + m) / 2 - t, (Q - P - m) / 2 + t, P - t])


def solve_scales_k_bruteforce(C11, C12, C22, n: int, grid: int = 20001):
    """Minimiser of kurtosis_objective_k over the feasible family by dense
    search refined with golden-section search (float64).  Slow; pins
    solve_scales_k_f32."""
    B = 12.0 / n
    M11, M12, M22 = B * C11, B * C12, B * C22
    P = (4 * M11 - M22) / 3.0
    Q = (4 * M22 - M11) / 3.0
    m = 2.5 * M12
    lo, hi = max(0.0, (P - Q + m) / 2), min(P, (P + Q + m) / 2)
    if hi <= lo:
        return scale_family_k(C11, C12, C22, n, lo)
    f = lambda t: kurtosis_objective_k(scale_family_k(C11, C12, C22, n, t))  # noqa: E731
    ts = np.linspace(lo, hi, grid)
    i = int(np.argmin([f(t) for t in ts]))
    a, b = ts[max(i - 1, 0)], ts[min(i + 1, grid - 1)]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        c, d = b - g * (b - a), a + g * (b - a)
        if f(c) < f(d):
            b = d
        else:
            a = c
    return scale_family_k(C11, C12, C22, n, 0.5 * (a + b))


# --------------------------------------------------------------------------
# The float32 solve the kernels decide in
# --------------------------------------------------------------------------

def solve_scales_k_f32(C11, C12, C22, n: int):
    """Minimum-kurtosis scales of beta'_a in float32, one fixed sequence of
    IEEE round-to-nearest operations (no fused multiply-add).

    Everything is carried times 3 (P3 = 3P, Q3 = 3Q, m3 = 3m, T = 3t), which
    keeps the divisions by 3 out; the depressed cubic keeps its form.
    1. Sanitise as params.solve_scales_f32: non-finite -> zero and BAD_FLAG,
       negative diagonals -> 0.
    2. M = B C (B = 12/n); P3 = 4 M11 - M22, Q3 = 4 M22 - M11, m3 = 7.5 M12.
    3. Beyond the bound: P3 < 0 -> 0, Q3 < 0 -> 0, |m3| > P3 + Q3 -> +-(P3 + Q3)
       (each sets CLAMP_FLAG).
    4. p3 = (50 (P3^2 + Q3^2) + 32 (P3 - Q3)^2 + 43 m3^2) / 400 (all terms
       >= 0), q3 = m3 (P3 - Q3) (P3 + Q3) / 32; V from -q3/p3 by two Newton
       steps (monotone on the concave side, q^2/p^3 <= 0.04 there: two steps
       reach float32 precision).
    5. T = (P3/2 + m3/4) + V clamped into [max(0, ((P3 - Q3) + m3)/2),
       min(P3, ((P3 + Q3) + m3)/2)]; 3A = (T, ((P3 + Q3) + m3)/2 - T,
       ((Q3 - P3) - m3)/2 + T, P3 - T), each floored at 0.
    Returns (3A[4, ...] float32, flags int32).
    """
    c11 = np.asarray(C11, dtype=_F)
    c12 = np.asarray(C12, dtype=_F)
    c22 = np.asarray(C22, dtype=_F)
    c11, c12, c22 = np.broadcast_arrays(c11, c12, c22)
    c11 = c11.copy(); c12 = c12.copy(); c22 = c22.copy()
    flags = np.zeros(c11.shape, dtype=np.int32)
    bad = ~(np.isfinite(c11) & np.isfinite(c12) & np.isfinite(c22))
    flags[bad] |= params.BAD_FLAG
    c11[bad] = 0; c12[bad] = 0; c22[bad] = 0
    c11 = np.fmax(c11, _F(0))
    c22 = np.fmax(c22, _F(0))
    B = _F(12.0) / _F(n)
    m11 = B * c11
    m22 = B * c22
    m12 = B * c12
    P3 = (_F(4) * m11 - m22).astype(_F)
    Q3 = (_F(4) * m22 - m11).astype(_F)
    m3 = (_F(7.5) * m12).astype(_F)
    negP, negQ = P3 < 0, Q3 < 0
    P3 = np.where(negP, _F(0), P3).astype(_F)
    Q3 = np.where(negQ, _F(0), Q3).astype(_F)
    S3 = (P3 + Q3).astype(_F)
    over = np.abs(m3) > S3
    m3 = np.where(over, np.copysign(S3, m3), m3).astype(_F)
    flags[negP | negQ | over] |= params.CLAMP_FLAG
    dPQ = (P3 - Q3).astype(_F)
    p = ((((_F(50) * ((P3 * P3) + (Q3 * Q3))) + (_F(32) * (dPQ * dPQ))) + (_F(43) * (m3 * m3)))
         / _F(400)).astype(_F)
    q = (((m3 * dPQ) * S3) * _F(0.03125)).astype(_F)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.where(p > 0, -q / np.where(p > 0, p, _F(1)), _F(0)).astype(_F)
        for _ in range(2):
            v2 = v * v
            h = (v2 + p) * v + q
            dh = _F(3.0) * v2 + p
            v = np.where(dh > 0, v - h / np.where(dh > 0, dh, _F(1)), v).astype(_F)
    T = ((_F(0.5) * P3 + _F(0.25) * m3) + v).astype(_F)
    half_sum = (_F(0.5) * (S3 + m3)).astype(_F)
    lo = np.fmax(_F(0.5) * (dPQ + m3), _F(0))
    hi = np.fmin(P3, half_sum)
    T = np.fmin(np.fmax(T, lo), hi).astype(_F)
    A3 = np.stack([np.fmax(T, _F(0)),
                   np.fmax(half_sum - T, _F(0)),
                   np.fmax(_F(0.5) * ((Q3 - P3) - m3) + T, _F(0)),
                   np.fmax(P3 - T, _F(0))]).astype(_F)
    return A3, flags


def steps_from_scales_k(A3, n: int, rule: str = "corrected"):
    """Continuous steps along e_k from 3A_k: lambda = sqrt(1 + 3A/15)
    ("corrected": L samples spaced sqrt(5) apart have variance A/12) or
    sqrt(3A/15) ("paper": the step scaling a/|e_k| of the running sums)."""
    A3 = np.asarray(A3, dtype=_F)
    r = (A3 / _F(15)).astype(_F)
    if rule == "corrected":
        lam = np.sqrt((_F(1) + r).astype(_F))
    elif rule == "paper":
        lam = np.sqrt(r)
    else:
        raise ValueError(rule)
    return lam.astype(_F)


def integer_steps_k(C11, C12, C22, n: int, rule: str = "corrected"):
    A3, flags = solve_scales_k_f32(C11, C12, C22, n)
    return params.round_steps(steps_from_scales_k(A3, n, rule), n), flags


def tap_extent_k(L, n: int):
    """(x_min, x_max, y_min, y_max) of the taps: along e_k the offsets run from
    -n(L_k+1)/2 to n(L_k-1)/2 (in units of e_k)."""
    L = np.asarray(L, dtype=np.int64)
    lo = -(n * (L + 1)) // 2
    hi = (n * (L - 1)) // 2
    x_max = 2 * hi[0] + hi[1] - lo[2] - 2 * lo[3]
    x_min = 2 * lo[0] + lo[1] - hi[2] - 2 * hi[3]
    y_max = hi[0] + 2 * hi[1] + 2 * hi[2] + hi[3]
    y_min = lo[0] + 2 * lo[1] + 2 * lo[2] + lo[3]
    return x_min, x_max, y_min, y_max


def reach_k(L, n: int):
    x_min, x_max, y_min, y_max = tap_extent_k(L, n)
    return np.maximum(np.maximum(-x_min, x_max), np.maximum(-y_min, y_max))


def realised_covariance_k(L, n: int) -> np.ndarray:
    """(n/12) sum_k (L_k^2 - 1) e_k e_k^T."""
    C = np.zeros((2, 2))
    for k, (ex, ey) in enumerate(DIRS_K):
        e = np.array([ex, ey], dtype=np.float64)
        C += n * (int(L[k]) ** 2 - 1) / 12.0 * np.outer(e, e)
    return C


# --------------------------------------------------------------------------
# Algorithm 3 in the integer-step form: running sums along e_k, then taps
# --------------------------------------------------------------------------

def _scan_k64(S: np.ndarray, ex: int, ey: int) -> None:
    """S(x, y) += S(x - ex, y - ey) in row order (S = 0 outside the domain)."""
    Hp, Wp = S.shape
    for y in range(ey, Hp):
        if ex >= 0:
            S[y, ex:] += S[y - ey, :Wp - ex]
        else:
            S[y, :Wp + ex] += S[y - ey, -ex:]


def _scan_k128(S: U128, ex: int, ey: int) -> None:
    Hp, Wp = S.lo.shape
    for y in range(ey, Hp):
        if ex >= 0:
            S[y, ex:] = S[y, ex:] + S[y - ey, :Wp - ex]
        else:
            S[y, :Wp + ex] = S[y, :Wp + ex] + S[y - ey, -ex:]


def preintegrate_k(fq_ext: np.ndarray, n: int, bits: int = 64):
    """n-fold running sums along e_1..e_4 (Algorithm 3, step 2, without the
    factor sqrt(5), which the normalisation absorbs), mod 2^bits (bits=32:
    the mod-2^64 sums reduced, as in modular.preintegrate)."""
    if bits == 32:
        with np.errstate(over="ignore"):
            return (preintegrate_k(fq_ext, n, 64) & U64(0xFFFFFFFF)).astype(np.uint32)
    if bits == 64:
        if fq_ext.dtype == object:
            S = np.vectorize(lambda v: int(v) & MASK64, otypes=[object])(fq_ext).astype(U64)
        else:
            S = fq_ext.astype(np.int64).view(U64).copy()
        with np.errstate(over="ignore"):
            for ex, ey in DIRS_K:
                for _ in range(n):
                    _scan_k64(S, ex, ey)
        return S
    if bits == 128:
        S = U128.from_ints(fq_ext.astype(object))
        for ex, ey in DIRS_K:
            for _ in range(n):
                _scan_k128(S, ex, ey)
        return S
    raise ValueError(bits)


def taps_k(S, Lfield: np.ndarray, n: int, R: int, H: int, W: int, bits: int = 64):
    """acc(p) = sum_t prod_k (-1)^t_k C(n, t_k) S(p + sum_k (c_k - t_k L_k) e_k)
    (bits=32: mod 2^32, read as a signed 32-bit value)."""
    if bits == 32:
        with np.errstate(over="ignore"):
            acc = taps_k(np.asarray(S).astype(U64), Lfield, n, R, H, W, 64)
        return (acc.view(U64) & U64(0xFFFFFFFF)).astype(np.uint32).view(np.int32).astype(np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    L = Lfield.astype(np.int64)
    c = (n * (L - 1)) // 2
    bx = xx + R
    by = yy + R
    for k, (ex, ey) in enumerate(DIRS_K):
        bx = bx + c[k] * ex
        by = by + c[k] * ey
    acc = np.zeros((H, W), dtype=U64) if bits == 64 else U128(np.zeros((H, W), U64), np.zeros((H, W), U64))
    with np.errstate(over="ignore"):
        for t in itertools.product(range(n + 1), repeat=4):
            w = 1
            tx, ty = bx, by
            for k, (ex, ey) in enumerate(DIRS_K):
                w *= (-1) ** t[k] * comb(n, t[k])
                tx = tx - t[k] * L[k] * ex
                ty = ty - t[k] * L[k] * ey
            g = S[ty, tx]
            if bits == 64:
                if w >= 0:
                    acc += U64(w) * g
                else:
                    acc -= U64(-w) * g
            else:
                for _ in range(abs(w)):
                    acc = acc + g if w > 0 else acc - g
    if bits == 64:
        return acc.view(np.int64)
    return acc.to_signed_ints()


def masses_k(Lfield: np.ndarray, n: int):
    H, W = Lfield.shape[1:]
    D = np.empty((H, W), dtype=object)
    for y in range(H):
        for x in range(W):
            D[y, x] = kernel_mass(Lfield[:, y, x], n)
    return D


def _steps_within(L, reach, R):
    far = reach > R
    return np.where(far[None], 1, L)


def filter_modular_k(f: np.ndarray, cov: np.ndarray, n: int, boundary: int, q: int,
                     bits: int = 64, out_dtype=np.float32, R: int | None = None,
                     rule: str = "corrected", return_all: bool = False):
    """Algorithm 3 with integer steps: beta'_a at every pixel."""
    H, W = f.shape
    L, flags = integer_steps_k(cov[0], cov[1], cov[2], n, rule)
    if R is None:
        R = max(int(reach_k(L, n).max(initial=0)), 3 * n)
    else:
        L = _steps_within(L, reach_k(L, n), R)
    fq = quantize(f, q, as_object=(bits == 128))
    S = preintegrate_k(extend_image(fq, R, boundary), n, bits)
    acc = taps_k(S, L, n, R, H, W, bits)
    D = masses_k(L, n)
    out = finalize(acc, D, q, out_dtype)
    if return_all:
        return dict(out=out, L=L, flags=flags, R=R, S=S, acc=acc, D=D)
    return out


def correlate_exact_k(fq, Lfield, n, boundary, pixels=None):
    """The definition for beta'_a: direct correlation with the kernel built on
    the lines Z e_k (kernels.correlate_exact with this direction set)."""
    return correlate_exact(fq, Lfield, n, boundary, pixels=pixels, dirs=DIRS_K)


# --------------------------------------------------------------------------
# Algorithm 2: the pair, switched per pixel by sector
# --------------------------------------------------------------------------

def use_knight(C11, C12, C22):
    """Sector S' test: |C11 - C22| < 3|C12| and |C12| < 2|C11 - C22|, with
    |C11 - C22| rounded once to float64 (inputs float32)."""
    c11 = np.asarray(C11, dtype=_F).astype(np.float64)
    c12 = np.asarray(C12, dtype=_F).astype(np.float64)
    c22 = np.asarray(C22, dtype=_F).astype(np.float64)
    d = np.abs(c11 - c22)
    a = np.abs(c12)
    return (d < 3.0 * a) & (a < 2.0 * d)


def pair_steps(cov: np.ndarray, n: int, rule: str = "corrected"):
    """(use_knight mask, steps of the chosen set, flags of the chosen set, reach)."""
    mask = use_knight(cov[0], cov[1], cov[2])
    L0, f0 = params.integer_steps(cov[0], cov[1], cov[2], n, rule)
    L1, f1 = integer_steps_k(cov[0], cov[1], cov[2], n, rule)
    L = np.where(mask[None], L1, L0)
    flags = np.where(mask, f1, f0)
    reach = np.where(mask, reach_k(L1, n), params.reach(L0, n))
    return mask, L, flags, reach


def algorithm2(f: np.ndarray, cov: np.ndarray, n: int, boundary: int, q: int, bits: int = 64,
               out_dtype=np.float32, R: int | None = None, rule: str = "corrected"):
    """Algorithm 2: both sets of running sums, and per pixel the finite
    differences of the set its sector picks.  Returns (out, mask, R)."""
    from . import modular
    mask, _, _, reach = pair_steps(cov, n, rule)
    if R is None:
        R = max(int(reach.max(initial=0)), 3 * n)
    out0 = modular.filter_modular(f, cov, n, boundary, q=q, bits=bits, out_dtype=out_dtype, R=R, rule=rule)
    out1 = filter_modular_k(f, cov, n, boundary, q=q, bits=bits, out_dtype=out_dtype, R=R, rule=rule)
    return np.where(mask, out1, out0), mask, R
