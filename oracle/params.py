"""Covariance / scale-vector geometry of the four-directional box spline.

Oracle module (test infrastructure only; see the package docstring).

Notation follows the paper: directions theta_k = 0, pi/4, pi/2, 3pi/4 with
grid vectors d_1 = (1,0), d_2 = (1,1), d_3 = (0,1), d_4 = (-1,1) (x is the
column, y the row), unit vectors u_k = d_k / |d_k|, scale vector
a = (a_1..a_4) and A_k = a_k^2 in px^2.  The order-n filter is the n-fold
self-convolution of beta_a.
"""
from __future__ import annotations

import math

import numpy as np

DIRS = ((1, 0), (1, 1), (0, 1), (-1, 1))
NORM2 = (1, 2, 1, 2)  # |d_k|^2


# --------------------------------------------------------------------------
# Geometry (Section 1.1, eq. "cov" and eq. "geometry")
# --------------------------------------------------------------------------

def covariance_of_scales(a, n: int = 1) -> np.ndarray:
    """Covariance of the n-fold box spline with scale vector a (float64).

    For n = 1 this is the paper's closed form (Section 1.1, the covariance
    matrix C_a):  (1/24) [[2a1^2 + a2^2 + a4^2, a2^2 - a4^2],
                          [a2^2 - a4^2, 2a3^2 + a2^2 + a4^2]].
    Covariances of symmetric unit-mass factors add (Proposition 1), so the
    n-fold self-convolution has n times that matrix.
    Pinned by tests: equals the second moments of the discrete impulse
    response in the integer-step limit, and sum_k a_k^2 u_k u_k^T / 12.
    """
    a = np.asarray(a, dtype=np.float64)
    a1, a2, a3, a4 = a[0] ** 2, a[1] ** 2, a[2] ** 2, a[3] ** 2
    c11 = 2 * a1 + a2 + a4
    c12 = a2 - a4
    c22 = 2 * a3 + a2 + a4
    return (n / 24.0) * np.array([[c11, c12], [c12, c22]])


def geometry_of_scales(a):
    """(size s, elongation rho, orientation theta) from eq. "geometry".

    s = (1/12) sum a_k^2, rho = (sum a_k^2 + sqrt(D)) / (sum a_k^2 - sqrt(D)),
    tan theta = (a3^2 - a1^2 + sqrt(D)) / (a2^2 - a4^2),
    D = (a1^2 - a3^2)^2 + (a2^2 - a4^2)^2.  theta is returned in [0, pi).
    Pinned by tests against the eigen-decomposition of covariance_of_scales.
    """
    a = np.asarray(a, dtype=np.float64)
    q = a ** 2
    tot = q.sum()
    D = (q[0] - q[2]) ** 2 + (q[1] - q[3]) ** 2
    s = tot / 12.0
    rho = (tot + math.sqrt(D)) / (tot - math.sqrt(D)) if tot > math.sqrt(D) else math.inf
    num = q[2] - q[0] + math.sqrt(D)
    den = q[1] - q[3]
    if den == 0.0:
        theta = 0.0 if num == 0.0 or q[0] >= q[2] else math.pi / 2
    else:
        theta = math.atan(num / den) % math.pi
    return s, rho, theta


def cov_from_sigma_rho_theta(sigma, rho, theta):
    """Covariance with trace 2 sigma^2, eigenvalue ratio rho, major axis at theta.

    Reading of the size/elongation/orientation parameterisation (Section 1.1:
    size = sum of eigenvalues, elongation = ratio of eigenvalues, orientation
    = angle of the top eigenvector); trace 2 sigma^2 makes rho = 1 give
    sigma^2 I.  Returns (C11, C12, C22) in float64.
    Pinned by tests against numpy.linalg.eigh.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    lam_min = 2.0 * sigma ** 2 / (1.0 + rho)
    lam_max = rho * lam_min
    c, s = np.cos(theta), np.sin(theta)
    return (lam_max * c * c + lam_min * s * s,
            (lam_max - lam_min) * c * s,
            lam_max * s * s + lam_min * c * c)


def elongation_bound(phi):
    """e(phi) of eq. "boundE": the largest elongation beta_a reaches at orientation phi.

    e = (1 + t + sqrt(1 + t^2)) / (1 + t - sqrt(1 + t^2)),
    t = |tan(phi) - cot(phi)| / 2.  Infinite on the four axes.
    Pinned by Table 4 ("previous bound" row) and by the feasibility edge of
    the scale solve.
    """
    phi = float(phi)
    s, c = math.sin(phi), math.cos(phi)
    if abs(s) < 1e-15 or abs(c) < 1e-15:
        return math.inf
    t = abs(s / c - c / s) / 2.0
    r = math.sqrt(1.0 + t * t)
    den = 1.0 + t - r
    return math.inf if den <= 0 else (1.0 + t + r) / den


def condition1_bound(C11, C12, C22):
    """Right side of eq. "condition1": the smallest eigenvalue of C."""
    return 0.5 * (C11 + C22 - math.sqrt((C11 - C22) ** 2 + 4 * C12 ** 2))


def condition2_bound(C11, C12, C22):
    """Right side of eq. "condition2", with phi the orientation of C.

    For an isotropic C the elongation term vanishes and the bound equals C11.
    """
    root = math.sqrt((C11 - C22) ** 2 + 4 * C12 ** 2)
    if root == 0.0:
        return 0.5 * (C11 + C22)
    lam_max = 0.5 * (C11 + C22 + root)
    phi = math.atan2(lam_max - C11, C12) if C12 != 0 else (0.0 if C11 >= C22 else math.pi / 2)
    e = elongation_bound(phi)
    ratio = 1.0 if math.isinf(e) else (e + 1.0) / (e - 1.0)
    return 0.5 * (C11 + C22 - ratio * root)


# --------------------------------------------------------------------------
# Minimum-kurtosis scale solve (Section 1.1 and the kurtosis matrix of
# Section 2.3, read for the Cartesian directions)
# --------------------------------------------------------------------------

def scale_family(C11, C12, C22, n: int, u):
    """The one-parameter family of A = a^2 with covariance C (float64).

    With B = 12/n, C = (n/12) sum_k A_k u_k u_k^T reads
    B C11 = A1 + (A2+A4)/2,  B C22 = A3 + (A2+A4)/2,  B C12 = (A2 - A4)/2,
    so with u = (A2 + A4)/2:  A1 = B C11 - u, A3 = B C22 - u,
    A2 = u + B C12, A4 = u - B C12, all >= 0 iff
    B |C12| <= u <= B min(C11, C22).
    """
    B = 12.0 / n
    return np.array([B * C11 - u, u + B * C12, B * C22 - u, u - B * C12])


def kurtosis_objective(A) -> float:
    """F = ||sum_k A_k^2 u_k u_k^T||_F^2 (the Frobenius-norm kurtosis criterion).

    The paper gives the kurtosis matrix of the rotated box spline as
    kappa sum_k a_k^4 u_k u_k^T (Section 2.3) and minimises its Frobenius norm;
    the Cartesian box spline is read the same way (parity of the reading
    unpinned beyond the isotropic solution a_k = sqrt(6) sigma).
    """
    A = np.asarray(A, dtype=np.float64)
    M = np.zeros((2, 2))
    for k, (dx, dy) in enumerate(DIRS):
        u = np.array([dx, dy], dtype=np.float64) / math.sqrt(NORM2[k])
        M += A[k] ** 2 * np.outer(u, u)
    return float((M * M).sum())


def solve_scales_bruteforce(C11, C12, C22, n: int, grid: int = 20001):
    """Minimiser of kurtosis_objective over the feasible family, by dense search
    refined with golden-section search in float64.  Slow; used only to pin
    solve_scales_f32."""
    B = 12.0 / n
    lo, hi = B * abs(C12), B * min(C11, C22)
    if hi <= lo:
        return scale_family(C11, C12, C22, n, lo)
    us = np.linspace(lo, hi, grid)
    Fs = np.array([kurtosis_objective(scale_family(C11, C12, C22, n, u)) for u in us])
    i = int(np.argmin(Fs))
    a, b = us[max(i - 1, 0)], us[min(i + 1, grid - 1)]
    g = (math.sqrt(5) - 1) / 2
    f = lambda u: kurtosis_objective(scale_family(C11, C12, C22, n, u))  # noqa: E731
    for _ in range(200):
        c, d = b - g * (b - a), a + g * (b - a)
        if f(c) < f(d):
            b = d
        else:
            a = c
    return scale_family(C11, C12, C22, n, 0.5 * (a + b))


CLAMP_FLAG = 1
BAD_FLAG = 2

_F = np.float32


def solve_scales_f32(C11, C12, C22, n: int):
    """Minimum-kurtosis scales A_k in float32, the precision the kernel decides in.

    The step sizes are integers rounded from these scales, so this solve is
    done in float32 with one fixed sequence of IEEE operations (no fused
    multiply-add), which any implementation can repeat bit for bit.

    Steps (arrays broadcast):
    1. Sanitise: non-finite input -> zero covariance and BAD_FLAG; negative
       diagonals -> 0; |C12| > min(C11, C22) (beyond the elongation bound
       e(phi)) -> C12 clamped to +-min(C11, C22) and CLAMP_FLAG.
    2. c1 = B C11, c3 = B C22, b = B C12 with B = 12/n.
    3. dF/du = 0 is the cubic 8u^3 - 6 s u^2 + (4(c1^2 + c3^2) + 8 b^2) u
       - (c1^3 + c3^3) - b^2 s (s = c1 + c3), which is strictly increasing.
       With u = s/4 + v it is v^3 + p v + q = 0, p = (2.5 d^2 + 2 c1 c3 + 8 b^2)/8,
       q = s (b^2 - d^2/4)/8, d = c1 - c3.  Newton's method from v0 = -q/p
       (an upper bound of the root's magnitude on the convex side) converges
       monotonically; v^2/p <= 0.16 at v0, and two steps already reach
       float32 precision (a third moves u by at most one unit in the last
       place), so two steps are taken.
    4. u is clamped into the feasible interval [|b|, min(c1, c3)] and
       A1 = c1 - u, A2 = u + b, A3 = c3 - u, A4 = u - b (each floored at 0).
       Minimum and maximum ignore a NaN operand (C fminf/fmaxf semantics).
    Returns (A[4, ...] float32, flags int32).
    Pinned by tests: against solve_scales_bruteforce, the isotropic closed form
    A_k = 6 sigma^2 / n, and covariance_of_scales(sqrt(A)) == C.
    """
    c11 = np.asarray(C11, dtype=_F)
    c12 = np.asarray(C12, dtype=_F)
    c22 = np.asarray(C22, dtype=_F)
    c11, c12, c22 = np.broadcast_arrays(c11, c12, c22)
    c11 = c11.copy(); c12 = c12.copy(); c22 = c22.copy()
    flags = np.zeros(c11.shape, dtype=np.int32)
    bad = ~(np.isfinite(c11) & np.isfinite(c12) & np.isfinite(c22))
    flags[bad] |= BAD_FLAG
    c11[bad] = 0; c12[bad] = 0; c22[bad] = 0
    c11 = np.fmax(c11, _F(0))
    c22 = np.fmax(c22, _F(0))
    m = np.fmin(c11, c22)
    over = np.abs(c12) > m
    flags[over] |= CLAMP_FLAG
    c12 = np.where(over, np.copysign(m, c12), c12).astype(_F)

    B = _F(12.0) / _F(n)
    c1 = B * c11
    c3 = B * c22
    b = B * c12
    s = c1 + c3
    d = c1 - c3
    bb = b * b
    dd = d * d
    p = ((_F(2.5) * dd + _F(2.0) * (c1 * c3)) + _F(8.0) * bb) * _F(0.125)
    q = (s * (bb - _F(0.25) * dd)) * _F(0.125)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.where(p > 0, -q / np.where(p > 0, p, _F(1)), _F(0)).astype(_F)
        for _ in range(2):
            v2 = v * v
            h = (v2 + p) * v + q
            dh = _F(3.0) * v2 + p
            v = np.where(dh > 0, v - h / np.where(dh > 0, dh, _F(1)), v).astype(_F)
    u = _F(0.25) * s + v
    lo = np.abs(b)
    hi = np.fmin(c1, c3)
    u = np.fmin(np.fmax(u, lo), hi)
    A = np.stack([np.fmax(c1 - u, _F(0)), np.fmax(u + b, _F(0)),
                  np.fmax(c3 - u, _F(0)), np.fmax(u - b, _F(0))]).astype(_F)
    return A, flags


L_MAX = 32767


def steps_from_scales(A, n: int, rule: str = "corrected"):
    """Continuous step lambda_k (in grid steps along d_k) from A_k, float32.

    "corrected" (default): lambda = sqrt(1 + A / |d|^2), so that L grid samples
    spaced |d| apart have variance |d|^2 (L^2 - 1)/12 = A/12, the variance a
    box of width a contributes along its direction.
    "paper": lambda = a / |d| = sqrt(A / |d|^2), the step scaling of the
    running sums (Section 1.1); it carries a -(n/12) sum_k |d_k|^2 d_k d_k^T
    covariance bias relative to the target.
    """
    A = np.asarray(A, dtype=_F)
    nrm = np.array([_F(1), _F(0.5), _F(1), _F(0.5)], dtype=_F).reshape((4,) + (1,) * (A.ndim - 1))
    if rule == "corrected":
        lam = np.sqrt(_F(1) + A * nrm)
    elif rule == "paper":
        lam = np.sqrt(A * nrm)
    else:
        raise ValueError(rule)
    return lam.astype(_F)


def round_steps(lam, n: int) -> np.ndarray:
    """Admissible integer step L nearest to lambda, ties to the larger value.

    Admissible: L >= 1, and L odd when n is odd (so the kernel centre
    n(L-1)/2 lies on the grid).  n odd: L = 2 floor(lambda/2) + 1;
    n even: L = floor(lambda + 1/2).  Capped at L_MAX.
    """
    lam = np.fmin(np.asarray(lam, dtype=_F), _F(L_MAX))
    if n % 2 == 1:
        L = _F(2) * np.floor(_F(0.5) * lam) + _F(1)
    else:
        L = np.floor(lam + _F(0.5))
    L = np.fmax(L, _F(1))
    return np.fmin(L, _F(L_MAX)).astype(np.int64)


def integer_steps(C11, C12, C22, n: int, rule: str = "corrected"):
    """Per-pixel integer steps L[4, ...] (int64) and flags from a covariance field."""
    A, flags = solve_scales_f32(C11, C12, C22, n)
    return round_steps(steps_from_scales(A, n, rule), n), flags


def tap_extent(L, n: int):
    """Offsets (x_min, x_max, y_min, y_max) spanned by the finite-difference taps.

    Tap t sits at sum_k (c_k - t_k L_k) d_k with c_k = n (L_k - 1)/2 and
    t_k in {0..n}: along d_k the offset runs from -n(L_k+1)/2 to n(L_k-1)/2.
    """
    L = np.asarray(L, dtype=np.int64)
    lo = -(n * (L + 1)) // 2
    hi = (n * (L - 1)) // 2
    x_min = lo[0] + lo[1] - hi[3]
    x_max = hi[0] + hi[1] - lo[3]
    y_min = lo[1] + lo[2] + lo[3]
    y_max = hi[1] + hi[2] + hi[3]
    return x_min, x_max, y_min, y_max


def reach(L, n: int):
    """Padding R needed so that every tap of every pixel lies in the padded domain."""
    x_min, x_max, y_min, y_max = tap_extent(L, n)
    return np.maximum(np.maximum(-x_min, x_max), np.maximum(-y_min, y_max))


def realised_covariance(L, n: int) -> np.ndarray:
    """Covariance of the integer-step kernel: (n/12) sum_k (L_k^2 - 1) d_k d_k^T."""
    C = np.zeros((2, 2))
    for k, (dx, dy) in enumerate(DIRS):
        d = np.array([dx, dy], dtype=np.float64)
        C += n * (int(L[k]) ** 2 - 1) / 12.0 * np.outer(d, d)
    return C
