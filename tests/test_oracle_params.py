"""Pins for oracle.params: geometry, scale solve, step rounding, e(phi)."""
import math

import numpy as np
import pytest

from oracle import params, gaussian
from tests.conftest import golden_rows


def test_isotropic_scales_closed_form():
    # Section 1.1: C_a = (a^2/6) I when all scales equal a, so a = sqrt(6) sigma
    # for n = 1; the n-fold filter needs A = 6 sigma^2 / n.
    for n in (1, 2, 3):
        for sig in (0.5, 1.0, 4.0, 16.0):
            A, fl = params.solve_scales_f32(sig * sig, 0.0, sig * sig, n)
            assert fl == 0
            np.testing.assert_allclose(A.ravel(), 6 * sig * sig / n, rtol=2e-7)


def test_covariance_of_scales_matches_fourier_hessian():
    # Independent route: the covariance is minus the Hessian of the box
    # spline's Fourier transform at w = 0.
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = rng.uniform(0.5, 5.0, size=4)
        h = 1e-3
        f = lambda wx, wy: gaussian.box_spline_ft(np.array(wx), np.array(wy), a, gaussian.CARTESIAN)  # noqa
        f0 = f(0.0, 0.0)
        hxx = (f(h, 0) - 2 * f0 + f(-h, 0)) / h ** 2
        hyy = (f(0, h) - 2 * f0 + f(0, -h)) / h ** 2
        hxy = (f(h, h) - f(h, -h) - f(-h, h) + f(-h, -h)) / (4 * h * h)
        C = params.covariance_of_scales(a, 1)
        np.testing.assert_allclose(C, -np.array([[hxx, hxy], [hxy, hyy]]), rtol=1e-4, atol=1e-6)


def test_geometry_matches_eigendecomposition():
    rng = np.random.default_rng(2)
    for _ in range(50):
        a = rng.uniform(0.2, 6.0, size=4)
        C = params.covariance_of_scales(a, 1)
        w, V = np.linalg.eigh(C)
        s, rho, th = params.geometry_of_scales(a)
        assert s == pytest.approx(w.sum(), rel=1e-12)
        assert rho == pytest.approx(w[1] / w[0], rel=1e-9)
        v = V[:, 1]
        th_ref = math.atan2(v[1], v[0]) % math.pi
        dth = abs(th - th_ref)
        assert min(dth, math.pi - dth) < 1e-7


def test_cov_from_sigma_rho_theta_eigen():
    rng = np.random.default_rng(3)
    for _ in range(50):
        sig, rho, th = rng.uniform(0.5, 20), rng.uniform(1, 6), rng.uniform(0, math.pi)
        c11, c12, c22 = params.cov_from_sigma_rho_theta(sig, rho, th)
        C = np.array([[c11, c12], [c12, c22]])
        w, V = np.linalg.eigh(C)
        assert w.sum() == pytest.approx(2 * sig * sig, rel=1e-12)
        assert w[1] / w[0] == pytest.approx(rho, rel=1e-9)
        if rho > 1.01:
            v = V[:, 1]
            t = math.atan2(v[1], v[0]) % math.pi
            d = abs(t - th)
            assert min(d, math.pi - d) < 1e-7


def test_scale_solve_satisfies_covariance_and_is_minimum_kurtosis():
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(120):
        sig, rho, th = rng.uniform(0.5, 24), rng.uniform(1, 5.5), rng.uniform(0, math.pi)
        n = int(rng.integers(1, 4))
        c = [np.float32(v) for v in params.cov_from_sigma_rho_theta(sig, rho, th)]
        A, fl = params.solve_scales_f32(*c, n)
        if fl:
            continue
        A = A.ravel().astype(np.float64)
        # constraint: the n-fold covariance of scales sqrt(A) equals C
        C = params.covariance_of_scales(np.sqrt(A), n)
        Cref = np.array([[c[0], c[1]], [c[1], c[2]]], dtype=np.float64)
        np.testing.assert_allclose(C, Cref, rtol=1e-5, atol=1e-5 * float(c[0] + c[2]))
        # minimality against a brute-force search of the objective
        Ab = params.solve_scales_bruteforce(float(c[0]), float(c[1]), float(c[2]), n, grid=1001)
        assert params.kurtosis_objective(A) <= params.kurtosis_objective(Ab) * (1 + 1e-5)
        np.testing.assert_allclose(A, Ab, rtol=1e-5, atol=1e-5 * Ab.max())
        checked += 1
    assert checked > 80


def test_feasibility_edge_is_the_elongation_bound():
    # The family is feasible iff |C12| <= min(C11, C22); the largest feasible
    # elongation at orientation phi must equal e(phi) of eq. "boundE".
    for deg in (5, 10, 13.3, 20, 22.5, 30, 35, 40, 55, 67.5, 80, 100, 112.5, 150):
        phi = math.radians(deg)
        lo, hi = 1.0, 200.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            c11, c12, c22 = params.cov_from_sigma_rho_theta(5.0, mid, phi)
            if abs(c12) <= min(c11, c22):
                lo = mid
            else:
                hi = mid
        assert lo == pytest.approx(params.elongation_bound(phi), rel=1e-6)


def test_elongation_bound_table4_previous_row():
    rows = golden_rows("table4_previous_bound.txt")
    assert len(rows) == 8
    for deg, printed, status in rows:
        e = params.elongation_bound(math.radians(float(deg)))
        if status == "ok":
            assert round(e, 1) == pytest.approx(float(printed), abs=0.051), deg
        else:
            # documented disagreement of the printed table with eq. "boundE"
            assert abs(e - float(printed)) > 0.2
    assert params.elongation_bound(math.radians(22.5)) == pytest.approx(5.83, abs=0.005)
    assert math.isinf(params.elongation_bound(0.0))


def test_condition_bounds():
    # isotropic: the elongation term vanishes and both bounds equal sigma^2
    assert params.condition2_bound(4.0, 0.0, 4.0) == pytest.approx(4.0)
    assert params.condition1_bound(4.0, 0.0, 4.0) == pytest.approx(4.0)
    c = params.cov_from_sigma_rho_theta(5.0, 3.0, math.pi / 8)
    assert params.condition2_bound(*c) < params.condition1_bound(*c)


def test_step_rule_integer_points_and_rounding():
    # lambda = sqrt(1 + A/|d|^2) is exactly L when A = |d|^2 (L^2 - 1)
    A = np.array([80.0, 2 * 48.0, 24.0, 2 * 8.0], dtype=np.float32).reshape(4, 1)
    lam = params.steps_from_scales(A, 1)
    np.testing.assert_array_equal(lam.ravel(), [9, 7, 5, 3])
    # admissible rounding: odd for odd n, ties to the larger
    lam = np.array([1.0, 1.99, 2.0, 2.5, 3.0, 3.99, 4.0, 9.85, 7.0], dtype=np.float32)
    np.testing.assert_array_equal(params.round_steps(lam, 1), [1, 1, 3, 3, 3, 3, 5, 9, 7])
    np.testing.assert_array_equal(params.round_steps(lam, 2), [1, 2, 2, 3, 3, 4, 4, 10, 7])
    # the worked isotropic example sigma = 4, n = 1: a = 9.80, L = (9, 7, 9, 7)
    L, fl = params.integer_steps(16.0, 0.0, 16.0, 1)
    assert list(L.ravel()) == [9, 7, 9, 7]
    np.testing.assert_allclose(params.realised_covariance(L.ravel(), 1), (176 / 12) * np.eye(2))


def test_clamp_and_bad_flags():
    A, fl = params.solve_scales_f32(np.float32(4.0), np.float32(5.0), np.float32(9.0), 1)
    assert fl == params.CLAMP_FLAG
    assert (A >= 0).all()
    A, fl = params.solve_scales_f32(np.float32(np.nan), np.float32(0), np.float32(1), 2)
    assert fl & params.BAD_FLAG
    np.testing.assert_array_equal(A.ravel(), 0)
    # zero covariance: identity filter
    L, fl = params.integer_steps(0.0, 0.0, 0.0, 3)
    assert list(L.ravel()) == [1, 1, 1, 1]


def test_reach_and_tap_extent():
    L = np.array([9, 7, 9, 7])
    xm, xM, ym, yM = params.tap_extent(L, 1)
    assert (xm, xM, ym, yM) == (-12, 11, -13, 10)
    assert params.reach(L, 1) == 13
