"""Pins for oracle.backward: the adjoint of the D1 filter."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import backward, kernels, modular, params
from oracle.rounding import quantize


def _field(H, W, seed, smax=3.0):
    return wl.random_cov_field(H, W, seed=seed, sigma_range=(0.3, smax), rho_range=(1.0, 3.5))


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
def test_adjoint_identity_exact(n, boundary):
    # <A f, g> = <f, A^T g> exactly for the integer operator (no 1/D):
    # forward accumulators of the running-sum pipeline against the modular adjoint
    H, W = 11, 14
    rng = np.random.default_rng(10 * n + boundary)
    f = rng.integers(-50, 50, size=(H, W)).astype(np.float64)
    g = rng.integers(-1000, 1000, size=(H, W)).astype(np.int64)
    cov = _field(H, W, seed=n)
    r = modular.filter_modular(f, cov, n, boundary, q=0, bits=64, out_dtype=np.float64, return_all=True)
    lhs = sum(int(a) * int(b) for a, b in zip(r["acc"].ravel(), g.ravel()))
    gacc = backward.adjoint_modular_acc(g, r["L"], n, boundary, r["R"])
    rhs = sum(int(a) * int(b) for a, b in zip(quantize(f, 0).ravel(), gacc.ravel()))
    assert lhs == rhs


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
def test_modular_adjoint_equals_explicit_scatter(n, boundary):
    H, W = 10, 13
    rng = np.random.default_rng(n + 7 * boundary)
    g = rng.integers(-10 ** 6, 10 ** 6, size=(H, W)).astype(np.int64)
    cov = _field(H, W, seed=3 + n)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    R = max(int(params.reach(L, n).max()), 3 * n)
    a = backward.adjoint_modular_acc(g, L, n, boundary, R)
    b = backward.adjoint_direct_acc(g, L, n, boundary)
    assert all(int(a[y, x]) == int(b[y, x]) for y in range(H) for x in range(W))


def test_adjoint_matches_finite_differences_of_the_forward():
    # the filter is linear in the image, so central differences of
    # L(f) = <out(f), gout> in float64 give the gradient exactly up to rounding
    H, W, n, boundary = 9, 11, 2, 2
    rng = np.random.default_rng(5)
    f = rng.normal(size=(H, W))
    gout = rng.normal(size=(H, W))
    cov = _field(H, W, seed=8)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    exact = backward.adjoint_f64(gout, L, n, boundary)
    eps = 1e-3
    for (y, x) in [(0, 0), (4, 5), (8, 10), (2, 9)]:
        fp, fm = f.copy(), f.copy()
        fp[y, x] += eps
        fm[y, x] -= eps
        lp = (kernels.correlate_f64(fp, L, n, boundary) * gout).sum()
        lm = (kernels.correlate_f64(fm, L, n, boundary) * gout).sum()
        assert (lp - lm) / (2 * eps) == pytest.approx(exact[y, x], rel=1e-8, abs=1e-10)
    # the fixed-point route agrees with the exact adjoint to float32 accuracy
    qg = backward.grad_frac_bits(np.abs(gout).max())
    fx = backward.adjoint_modular(gout.astype(np.float32), L, n, boundary, qg,
                                  max(int(params.reach(L, n).max()), 3 * n))
    np.testing.assert_allclose(fx, exact, rtol=1e-5, atol=1e-5 * np.abs(exact).max())


def test_grad_frac_bits():
    assert backward.grad_frac_bits(1.0) == 54
    assert backward.grad_frac_bits(1.5) == 53
    assert backward.grad_frac_bits(0.5) == 55
    assert backward.grad_frac_bits(0.0) == 54
    assert backward.grad_frac_bits(2.0 ** 60) == 0


def test_grad_frac_bits_wide():
    assert backward.grad_frac_bits_wide(1.0) == 118
    assert backward.grad_frac_bits_wide(1.5) == 117
    assert backward.grad_frac_bits_wide(2.0 ** -20) == 126
    assert backward.grad_frac_bits_wide(2.0 ** 120) == 0


def test_wide_format_keeps_large_kernels_accurate():
    # kernel masses near 2^60 (n = 3, steps ~ 40): the 64-bit format's weights
    # 2^54 gout / D round to a few units and lose the gradient, the 128-bit
    # format keeps it to float32 accuracy against the float64 adjoint
    H, W, n, boundary = 7, 9, 3, 2
    rng = np.random.default_rng(11)
    gout = rng.normal(size=(H, W)).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=12, sigma_range=(24.0, 28.0), rho_range=(1.0, 2.0))
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    assert max(kernels.kernel_mass(L[:, y, x], n) for y in range(H) for x in range(W)) > 2 ** 55
    exact = backward.adjoint_f64(gout.astype(np.float64), L, n, boundary)
    wide = backward.adjoint_direct_wide(gout, L, n, boundary)
    scale = np.abs(exact).max()
    np.testing.assert_allclose(wide, exact, rtol=2e-6, atol=2e-6 * scale)
    narrow = backward.adjoint_direct(gout, L, n, boundary, backward.grad_frac_bits(np.abs(gout).max()))
    assert np.abs(narrow - exact).max() > 1e-3 * scale
