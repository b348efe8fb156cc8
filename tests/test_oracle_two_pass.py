"""Pins of Algorithm 1's oracle (oracle/two_pass.py): the algebraic
condition-2 bound against the trigonometric one, the isotropic closed form,
the validity of the residual covariance, Proposition 1 for the composed
passes (impulse response covariance = sum of the two realised covariances),
and the continuous-model accuracy of the split against Tables 2 and 3."""
import math

import numpy as np

from oracle import gaussian, kernels, modular, params
from oracle import two_pass as tp
from tests.conftest import golden_rows
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


def _split_errors(s, rho, theta, frac, dw=0.04):
    """Normalised L2 errors (Section 3) of the BoxFilter and of Algorithm 1 for
    one target, the split taken by this module on a one-pixel field: the
    min-kurtosis scales of C, then sqrt(6) sigma0 and the min-kurtosis scales
    of the residual (n = 1: A_k are the squared scales)."""
    C = np.array(params.cov_from_sigma_rho_theta(math.sqrt(s / 2.0), rho, theta), dtype=np.float64)
    field = np.asarray(C, dtype=np.float32).reshape(3, 1, 1)
    s2 = tp.sigma2_global(field, frac)
    iso, res = tp.split_field(field, s2)

    def scales(c):
        A, flags = params.solve_scales_f32(c[0, 0, 0], c[1, 0, 0], c[2, 0, 0], 1)
        assert int(flags) == 0
        return [math.sqrt(float(a)) for a in np.asarray(A).ravel()]

    target = np.array([[C[0], C[1]], [C[1], C[2]]])
    e_box = gaussian.normalized_l2_error([(scales(field), gaussian.CARTESIAN)], target, dw=dw)
    e_alg1 = gaussian.normalized_l2_error([(gaussian.isotropic_scales(math.sqrt(float(s2))), gaussian.CARTESIAN),
                                           (scales(res), gaussian.CARTESIAN)], target, dw=dw)
    return e_box, e_alg1


def test_table2_isotropic_columns_through_the_split():
    # the isotropic columns of Table 2 again, now through sigma2_global and
    # split_field instead of the closed form sigma0^2 = sigma^2 / 2
    for name, box_pct, alg1_pct in golden_rows("table2_isotropic.txt"):
        s = float(name.strip("()").split(",")[0])
        e_box, e_alg1 = _split_errors(s, 1.0, 0.0, 0.5, dw=0.02)
        assert round(100 * e_box, 1) == float(box_pct)
        assert round(100 * e_alg1, 1) == float(alg1_pct)


def test_table3_improvement_peaks_near_half_the_bound():
    # Table 3's shape.  Its values are not reproduced: with this module's
    # kurtosis reading the BoxFilter error of this target is 18.1 % and the
    # improvements run 16-39 % against the printed 3.5-33.3 %.  What holds:
    # the improvement grows from 10 % to 50 % of the bound, peaks at 50-60 %
    # (the printed 33.3 and 33.13 differ by 0.2 points; here by 0.6) and falls
    # beyond.
    rows = golden_rows("table3_sigma_fraction.txt")
    pct = [int(r[0]) for r in rows]
    printed = [float(r[1]) for r in rows]
    got = []
    for p in pct:
        e_box, e_alg1 = _split_errors(5.0, 3.0, math.pi / 4, p / 100.0)
        got.append(100 * (e_box - e_alg1) / e_box)
    for seq in (printed, got):
        i50, i60 = pct.index(50), pct.index(60)
        assert all(seq[i] < seq[i + 1] for i in range(i50))           # rising up to 50 %
        assert max(seq) in (seq[i50], seq[i60]) and abs(seq[i50] - seq[i60]) < 1.0
        assert all(seq[i] > seq[i + 1] for i in range(i60, len(seq) - 1))  # falling after 60 %
    assert all(g > 0 for g in got)
