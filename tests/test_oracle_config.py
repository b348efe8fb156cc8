"""Pins for oracle.config: the padding, mass bound and automatic q that the
GPU tests check the library's configuration against."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as wl
from oracle import config, continuous, kernels, params


def _tap_offsets(L, n):
    """Every tap offset sum_k (c_k - t_k L_k) d_k, t in {0..n}^4, by enumeration."""
    out = []
    for t in itertools.product(range(n + 1), repeat=4):
        x = y = 0
        for k, (dx, dy) in enumerate(params.DIRS):
            o = n * (L[k] - 1) // 2 - t[k] * L[k]
            x += o * dx
            y += o * dy
        out.append((x, y))
    return out


@pytest.mark.parametrize("n", [1, 2, 3])
def test_padding_covers_every_tap_and_is_tight(n):
    cov = wl.random_cov_field(9, 11, seed=n, sigma_range=(0.3, 7.0), rho_range=(1.0, 4.0))
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    brute = 3 * n
    for y in range(9):
        for x in range(11):
            offs = _tap_offsets([int(v) for v in L[:, y, x]], n)
            brute = max(brute, max(max(abs(a), abs(b)) for a, b in offs))
    assert config.padding(cov, n) == brute


@pytest.mark.parametrize("n", [1, 2])
def test_continuous_reach_field_equals_per_pixel_reach(n):
    planes = wl.param_fields_logsig_theta_logrho(7, 10, 3, logsig_range=(-1.0, 2.5), logrho_range=(0.0, 1.1))
    C = continuous.covariance_planes(planes, 1)
    Hs, _, _ = continuous.half_steps(*C, n)
    field = config.continuous_reach(Hs, n)
    for y in range(7):
        for x in range(10):
            assert field[y, x] == continuous.reach_d2(Hs[:, y, x], n)
    # identity steps reach 9 (n = 2) or 6 (n = 1): the floor of the padding
    ident = np.full((4, 1, 1), continuous.HALF)
    assert config.continuous_reach(ident, n)[0, 0] == (9 if n == 2 else 6)


def test_masses_are_the_kernel_masses():
    rng = np.random.default_rng(2)
    L = rng.integers(1, 9, size=(4, 5, 6))
    for n in (1, 2, 3):
        m = config.integer_masses_f32(L, n)
        for y in range(5):
            for x in range(6):
                assert m[y, x] == np.float32(kernels.kernel_mass(L[:, y, x], n))
    Hs = rng.integers(512, 5000, size=(4, 3, 3))
    for n in (1, 2):
        m = config.continuous_masses_f32(Hs, n)
        for y in range(3):
            for x in range(3):
                exact = math.prod(sum(continuous.line_kernel(continuous.line_taps(int(h), n)[0], n)[0])
                                  for h in Hs[:, y, x])
                assert abs(float(m[y, x]) - exact) <= 4 * 2.0 ** -24 * exact


@pytest.mark.parametrize("bits", [32, 64, 128])
def test_automatic_q_is_the_largest_with_one_guard_bit(bits):
    # (vmax 2^q + 1/2) mass < 2^(b-2) holds at the chosen q and fails two bits higher
    rng = np.random.default_rng(bits)
    for _ in range(400):
        vmax = float(np.float32(math.exp(rng.uniform(-8, 12))))
        mass = float(np.float32(math.exp(rng.uniform(0, 40))))
        q = config.auto_frac_bits(vmax, mass, bits)
        cap = 30 if bits == 32 else bits - 28
        lim = Fraction(2) ** (bits - 2)
        if q < cap:
            assert (Fraction(vmax) * Fraction(2) ** (q + 2)) * Fraction(mass) >= lim
        if q >= 0 and mass < 2.0 ** (bits - 2):   # (beyond it no q fits: the stencil flags overflow)
            assert (Fraction(vmax) * Fraction(2) ** q + Fraction(1, 2)) * Fraction(mass) < lim
        assert config.auto_frac_bits(vmax, mass, bits, continuous=True) == min(q, cap) - 2 or q >= cap


def test_automatic_width():
    img8 = np.zeros((2, 2), np.uint8)
    imgf = np.full((2, 2), 3.0, np.float32)
    # 8-bit images take 32 bits while q = 0 fits; float images need q >= 25 - ceil(log2 max)
    assert config.resolve(img8, 2.0 ** 20, -1, None) == (32, 1)
    assert config.resolve(img8, 2.0 ** 23, -1, None)[0] == 64
    assert config.resolve(imgf, 2.0 ** 10, -1, None)[0] == 64
    assert config.resolve(imgf, 2.0 ** 40, -1, None)[0] == 128
    assert config.resolve(imgf, 2.0 ** 10, -1, None, continuous=True)[0] == 64
    assert config.resolve(img8, 2.0 ** 8, 40, None) == (64, 40)
    assert config.resolve(img8, 2.0 ** 20, 40, None) == (128, 40)
