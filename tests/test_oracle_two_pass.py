"""Pins of Algorithm 1's oracle (oracle/two_pass.py): the algebraic
condition-2 bound against the trigonometric one, the isotropic closed form,
the validity of the residual covariance, and Proposition 1 for the composed
passes (impulse response covariance = sum of the two realised covariances)."""
import math

import numpy as np

from oracle import kernels, modular, params
from oracle import two_pass as tp
from workloads import synth


def test_condition2_algebraic_equals_trigonometric():
    rng = np.random.default_rng(0)
    for _ in range(500):
        s, rho, th = rng.uniform(0.5, 10), rng.uniform(1, 5.5), rng.uniform(0, math.pi)
        C = [float(c) for c in params.cov_from_sigma_rho_theta(s, rho, th)]
        a, b = tp.condition2_bound(*C), params.condition2_bound(*C)
        assert abs(a - b) <= 1e-10 * max(abs(b), 1.0)
    assert tp.condition2_bound(4.0, 0.0, 4.0) == 4.0      # isotropic: sigma^2
    assert tp.condition2_bound(5.0, 0.0, 2.0) == 2.0      # on an axis: the smallest eigenvalue


def test_isotropic_field_takes_half_its_variance():
    cov = synth.constant_cov_field(8, 9, 6.25, 0.0, 6.25)
    assert tp.sigma2_global(cov) == np.float32(3.125)
    iso, res = tp.split_field(cov, tp.sigma2_global(cov))
    assert (iso[0] == np.float32(3.125)).all() and (iso[1] == 0).all()
    assert (res[0] == np.float32(3.125)).all() and (res[2] == np.float32(3.125)).all()


def test_residual_stays_within_the_elongation_bound():
    # with sigma^2 below the condition-2 bound the residual needs no clamping
    cov = synth.random_cov_field(40, 40, seed=3, sigma_range=(1.0, 8.0), rho_range=(1.0, 5.0))
    s2 = tp.sigma2_global(cov)
    assert s2 > 0
    _, res = tp.split_field(cov, s2)
    _, flags = params.solve_scales_f32(res[0], res[1], res[2], 2)
    assert not (flags & params.CLAMP_FLAG).any()


def test_two_passes_add_covariances():
    # Proposition 1 on the composed filters: the impulse response of the two
    # passes has the covariance of the first pass's integer steps plus the
    # second's, up to the float32 rounding between the passes
    H = W = 81
    n = 2
    cov = synth.constant_cov_field(H, W, 7.0, 1.5, 5.0)
    s2 = tp.sigma2_global(cov)
    iso, res = tp.split_field(cov, s2)
    L_iso, _ = params.integer_steps(iso[0, 0, 0], iso[1, 0, 0], iso[2, 0, 0], n)
    L_res, _ = params.integer_steps(res[0, 0, 0], res[1, 0, 0], res[2, 0, 0], n)
    R = int(params.reach(L_iso.ravel(), n)) + int(params.reach(L_res.ravel(), n)) + 3 * n
    f = np.zeros((H, W))
    f[40, 40] = 1.0
    out, _, _ = tp.algorithm1(f, cov, n, kernels.ZERO, q=40, R=R, bits=128, out_dtype=np.float64)
    ys, xs = np.mgrid[0:H, 0:W]
    X, Y = xs - 40, ys - 40
    m = out.sum()
    got = np.array([[(out * X * X).sum(), (out * X * Y).sum()], [(out * X * Y).sum(), (out * Y * Y).sum()]]) / m
    want = params.realised_covariance(L_iso.ravel(), n) + params.realised_covariance(L_res.ravel(), n)
    assert abs(m - 1.0) < 1e-6
    assert np.allclose(got, want, atol=1e-4)


def test_zero_sigma_reduces_to_one_pass():
    # a field at the elongation bound somewhere leaves no room for the
    # isotropic pass: sigma^2 = 0, the first pass is the identity
    H, W = 12, 10
    cov = synth.constant_cov_field(H, W, 4.0, 4.0, 4.0)   # |C12| = min(C11, C22): bound 0 or below
    assert tp.sigma2_global(cov) == 0
    f = synth.random_integer_image(H, W, seed=1).astype(np.float32)
    out, _, g = tp.algorithm1(f, cov, 1, kernels.SYMMETRIC, q=8, R=20)
    np.testing.assert_array_equal(g, f)
    np.testing.assert_array_equal(out, modular.filter_modular(f, cov, 1, kernels.SYMMETRIC, q=8, R=20))
