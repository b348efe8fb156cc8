"""Pins the integer steps of the float32 step solve to the float64 minimiser.

The library and oracle.params decide every pixel's steps in float32 (two
Newton steps on the stationarity cubic, one fixed sequence of IEEE
operations, Section 1.1's minimum-kurtosis choice read with Section 2.3's
kurtosis matrix).  These tests check that choice against the exact minimiser
of the objective, found here in float64 without the cubic: bisection on the
derivative of F(u) = ||sum_k A_k(u)^2 u_k u_k^T||_F^2 along the feasible
family, the derivative written from the definition of F.  A step may differ
from the float64 one only where the float64 lambda lies within a stated
distance of a rounding boundary of the step rule; the number of such pixels
is printed.

The same holds for the covariance encoding of the log-parameter planes
(float32 exp and sin/cos) against the float64 formula, at the level of the
integer steps L (D1) and of the quantised steps H = RNE(512 lambda) (D2).
"""
import math

import numpy as np
import pytest

from oracle import continuous as cn
from oracle import params

NORM2 = np.array(params.NORM2, dtype=np.float64).reshape(4, 1)


def _unit_outer():
    out = []
    for dx, dy in params.DIRS:
        u = np.array([dx, dy], dtype=np.float64) / math.hypot(dx, dy)
        out.append(np.outer(u, u))
    return np.array(out)                                  # [4][2][2]


UU = _unit_outer()


def _family(c1, c3, b, u):
    # A_k along the feasible line: the covariance constraint fixes
    # A1 + A2/2 + A4/2 = c1, A3 + A2/2 + A4/2 = c3, (A2 - A4)/2 = b
    return np.stack([c1 - u, u + b, c3 - u, u - b])


def _dF(c1, c3, b, u):
    """dF/du from F = sum_ij M_ij^2 with M = sum_k A_k^2 u_k u_k^T and
    dA/du = (-1, 1, -1, 1): dF/du = sum_ij 2 M_ij sum_k 2 A_k dA_k/du (u_k u_k^T)_ij."""
    A = _family(c1, c3, b, u)
    M = np.einsum("kp,kij->pij", A * A, UU)
    sgn = np.array([-1.0, 1.0, -1.0, 1.0]).reshape(4, 1)
    dM = np.einsum("kp,kij->pij", 2.0 * A * sgn, UU)
    return 2.0 * (M * dM).sum(axis=(1, 2))


def solve_f64(C11, C12, C22, n):
    """Minimiser A_k (float64) of F over the feasible family, by bisection on
    dF/du (F is convex along the family), after the documented sanitising:
    negative diagonals to 0, C12 clamped to +-min(C11, C22)."""
    c11 = np.fmax(np.asarray(C11, np.float64), 0.0)
    c22 = np.fmax(np.asarray(C22, np.float64), 0.0)
    m = np.fmin(c11, c22)
    c12 = np.asarray(C12, np.float64)
    c12 = np.where(np.abs(c12) > m, np.copysign(m, c12), c12)
    B = 12.0 / n
    c1, c3, b = B * c11, B * c22, B * c12
    lo, hi = np.abs(b), np.fmin(c1, c3)
    a, z = lo.copy(), hi.copy()
    for _ in range(64):       # 2^-64 of the interval: below float64 resolution
        mid = 0.5 * (a + z)
        pos = _dF(c1, c3, b, mid) > 0
        z = np.where(pos, mid, z)
        a = np.where(pos, a, mid)
    u = 0.5 * (a + z)
    return np.fmax(_family(c1, c3, b, u), 0.0)


def lam_f64(A, rule):
    return np.sqrt(1.0 + A / NORM2) if rule == "corrected" else np.sqrt(A / NORM2)


def round_f64(lam, n):
    if n % 2:
        L = 2.0 * np.floor(0.5 * lam) + 1.0
    else:
        L = np.floor(lam + 0.5)
    return np.fmax(L, 1.0).astype(np.int64)


def boundary_distance(lam, n):
    """Distance of lambda to the nearest rounding boundary of the step rule:
    the half-integers for even n, the even integers for odd n."""
    if n % 2:
        return np.abs(lam - 2.0 * np.rint(0.5 * lam))
    return np.abs(lam - (np.floor(lam) + 0.5))


def covariance_sample(count, seed):
    """float32 (C11, C12, C22) mixing the cases where a float32 solve could
    drift: general, near-isotropic, within 1e-3 of the e(phi) edge, clamped
    (beyond the edge), axis-aligned, exactly isotropic, and tiny."""
    rng = np.random.default_rng(seed)
    k = count // 7
    parts = []
    sig = np.exp(rng.uniform(math.log(0.3), math.log(40.0), k))
    parts.append(params.cov_from_sigma_rho_theta(sig, rng.uniform(1, 5.8, k), rng.uniform(0, math.pi, k)))
    sig = np.exp(rng.uniform(math.log(0.3), math.log(40.0), k))
    parts.append(params.cov_from_sigma_rho_theta(sig, 1 + rng.uniform(0, 1e-3, k), rng.uniform(0, math.pi, k)))
    for shrink in (lambda m: m * (1 - rng.uniform(0, 1e-3, k)), lambda m: m * (1 + rng.uniform(0, 0.5, k))):
        c11 = rng.uniform(0.1, 400.0, k)
        c22 = c11 * np.exp(rng.uniform(-2.5, 2.5, k))
        m = shrink(np.fmin(c11, c22))
        parts.append((c11, m * rng.choice([-1.0, 1.0], k), c22))
    c11 = rng.uniform(0.1, 400.0, k)
    parts.append((c11, np.zeros(k), c11 * np.exp(rng.uniform(-2, 2, k))))
    c = rng.uniform(0.05, 600.0, k)
    parts.append((c, np.zeros(k), c))
    sig = rng.uniform(0.0, 0.7, count - 6 * k)
    parts.append(params.cov_from_sigma_rho_theta(sig, rng.uniform(1, 4, sig.size), rng.uniform(0, math.pi, sig.size)))
    return tuple(np.concatenate([p[i] for p in parts]).astype(np.float32) for i in range(3))


# distance (relative to lambda) within which a float32 decision may differ from
# the float64 one: the solve's scales carry a few float32 units of error
# (2 Newton steps reach 1.2e-7 relative), lambda a few more; 2^-18 leaves a
# margin of about 20x
REL_TOL = 2.0 ** -18


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("rule", ["corrected", "paper"])
def test_float32_steps_equal_float64_minimiser_away_from_boundaries(n, rule):
    C11, C12, C22 = covariance_sample(105_000, seed=100 + n)
    L32, _ = params.integer_steps(C11, C12, C22, n, rule)
    A64 = solve_f64(C11.astype(np.float64), C12.astype(np.float64), C22.astype(np.float64), n)
    lam = lam_f64(A64, rule)
    L64 = np.minimum(round_f64(lam, n), params.L_MAX)
    diff = L32 != L64
    dist = boundary_distance(lam, n)
    print(f"n={n} {rule}: {int(diff.sum())} of {diff.size} steps differ from the float64 minimiser's, "
          f"all within {dist[diff].max(initial=0) / max(lam[diff].max(initial=1), 1):.2e} (relative) "
          "of a rounding boundary")
    assert (dist[diff] <= REL_TOL * np.fmax(lam[diff], 1.0)).all()
    assert (np.abs(L32 - L64) <= 2).all()
    assert diff.sum() <= 1e-3 * diff.size


@pytest.mark.parametrize("n", [1, 2, 3])
def test_float32_scales_near_float64_minimiser(n):
    # the scales themselves, away from the integer decision: each A_k within
    # 2e-6 of the family's scale 12 max(C11, C22)/n
    C11, C12, C22 = covariance_sample(70_000, seed=7 + n)
    A32, _ = params.solve_scales_f32(C11, C12, C22, n)
    A64 = solve_f64(C11.astype(np.float64), C12.astype(np.float64), C22.astype(np.float64), n)
    scale = 12.0 / n * np.fmax(C11, C22).astype(np.float64)
    err = np.abs(A32.astype(np.float64) - A64) / np.fmax(scale, 1e-30)
    assert err.max() < 2e-6


def test_bisection_minimiser_matches_brute_force():
    # the float64 minimiser used above against the dense search of the objective
    rng = np.random.default_rng(5)
    for _ in range(12):
        sig, rho, th = rng.uniform(0.5, 9), rng.uniform(1, 5.5), rng.uniform(0, math.pi)
        C = params.cov_from_sigma_rho_theta(sig, rho, th)
        for n in (1, 2):
            ref = params.solve_scales_bruteforce(*C, n, grid=4001)
            A = solve_f64(np.array([C[0]]), np.array([C[1]]), np.array([C[2]]), n)[:, 0]
            np.testing.assert_allclose(A, ref, rtol=0, atol=1e-6 * 12 / n * max(C[0], C[2]))


# the log-parameter encoding: float32 exp and sin/cos against float64 (its
# relative error reaches a few 1e-7 of sigma^2, which moves lambda by about
# the same relative amount; near the elongation edge a small scale can
# carry a larger relative error, so the distance is taken against the
# largest lambda of the pixel)
LOG_REL_TOL = 2.0 ** -15


def _log_planes(count, seed):
    rng = np.random.default_rng(seed)
    ls = rng.uniform(-1.0, 3.5, count).astype(np.float32)
    th = rng.uniform(-0.5, 3.7, count).astype(np.float32)
    lr = rng.uniform(0.0, 1.7, count).astype(np.float32)
    return ls, th, lr


def _cov64(ls, th, lr):
    return params.cov_from_sigma_rho_theta(np.exp(ls.astype(np.float64)), np.exp(lr.astype(np.float64)),
                                           th.astype(np.float64))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_log_parameter_encoding_integer_steps(n):
    ls, th, lr = _log_planes(120_000, seed=40 + n)
    C32 = cn.cov_from_log_params(ls, th, lr)
    L32, _ = params.integer_steps(*C32, n)
    lam = lam_f64(solve_f64(*_cov64(ls, th, lr), n), "corrected")
    L64 = np.minimum(round_f64(lam, n), params.L_MAX)
    diff = (L32 != L64).any(axis=0)
    dist = boundary_distance(lam, n)
    near = dist <= LOG_REL_TOL * lam.max(axis=0)
    print(f"n={n}: {int(diff.sum())} of {diff.size} pixels with a step unlike the float64 encoding's")
    assert (near | (L32 == L64)).all()
    assert diff.sum() <= 2e-3 * diff.size


@pytest.mark.parametrize("n", [1, 2])
def test_log_parameter_encoding_quantised_steps(n):
    # D2: H = RNE(512 lambda), boundaries at (k + 1/2) / 512
    ls, th, lr = _log_planes(60_000, seed=60 + n)
    C32 = cn.cov_from_log_params(ls, th, lr)
    H32, _, _ = cn.half_steps(*C32, n)
    lam = lam_f64(solve_f64(*_cov64(ls, th, lr), n), "corrected")
    x = lam * cn.HALF
    H64 = np.minimum(np.rint(x).astype(np.int64), cn.H_MAX)
    dist = np.abs(x - (np.floor(x) + 0.5))           # in units of 2^-9
    diff = H32 != H64
    near = dist <= LOG_REL_TOL * x.max(axis=0)
    print(f"n={n}: {int(diff.any(axis=0).sum())} of {diff.shape[1]} pixels with a quantised step unlike "
          "the float64 encoding's")
    assert (near | ~diff).all()
    assert (np.abs(H32 - H64) <= 1).all()
