"""Pins for oracle.kernels and oracle.modular (the two oracle modes)."""
import itertools

import numpy as np
import pytest
import scipy.ndimage as ndi

import workloads as wl
from oracle import params, kernels, modular
from oracle.rounding import quantize, rn_f32_int, _rn32_array, finalize


def test_box_power_closed_forms():
    for L in (1, 2, 3, 5, 8):
        for n in (1, 2, 3):
            h = np.array(kernels.box_power_1d(L, n), dtype=np.float64)
            assert h.sum() == L ** n
            np.testing.assert_array_equal(h, h[::-1])
            j = np.arange(len(h)) - (len(h) - 1) / 2
            assert (h * j * j).sum() / h.sum() == pytest.approx(n * (L * L - 1) / 12)
        # n = 2 is the discrete triangle L - |j|
        h2 = np.array(kernels.box_power_1d(L, 2))
        j = np.arange(-(L - 1), L)
        np.testing.assert_array_equal(h2, L - np.abs(j))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_kernel_mass_symmetry_covariance(n):
    rng = np.random.default_rng(n)
    for _ in range(6):
        L = tuple(int(v) for v in rng.integers(1, 6, size=4))
        if n % 2 == 1:
            L = tuple(2 * (v // 2) + 1 for v in L)
        K, ox, oy = kernels.kernel_d1(L, n)
        Kf = K.astype(np.float64)
        assert int(K.sum()) == kernels.kernel_mass(L, n)
        assert (Kf >= 0).all()
        np.testing.assert_array_equal(Kf, Kf[::-1, ::-1])          # K(j) = K(-j)
        assert (oy, ox) == ((K.shape[0] - 1) // 2, (K.shape[1] - 1) // 2)
        yy, xx = np.mgrid[0:K.shape[0], 0:K.shape[1]]
        dx, dy = xx - ox, yy - oy
        m = Kf.sum()
        C = np.array([[(Kf * dx * dx).sum(), (Kf * dx * dy).sum()],
                      [(Kf * dx * dy).sum(), (Kf * dy * dy).sum()]]) / m
        # Proposition 1: covariances of the four symmetric unit-mass line kernels add
        np.testing.assert_allclose(C, params.realised_covariance(L, n), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("boundary,mode", [(kernels.ZERO, "constant"),
                                           (kernels.REPLICATE, "nearest"),
                                           (kernels.SYMMETRIC, "reflect")])
def test_axis_only_kernel_is_repeated_uniform_filter(boundary, mode):
    # L2 = L4 = 1: the kernel is separable boxes along x and y; compare with
    # scipy.ndimage.uniform_filter applied n times (odd sizes: centred boxes).
    H, W = 11, 14
    f = wl.random_integer_image(H, W, seed=5, lo=0, hi=50)
    for n, L1, L3 in [(1, 5, 3), (2, 3, 5), (3, 3, 1), (2, 7, 7)]:
        Lf = np.zeros((4, H, W), dtype=np.int64)
        Lf[0], Lf[1], Lf[2], Lf[3] = L1, 1, L3, 1
        out = kernels.correlate_f64(f, Lf, n, boundary)
        ref = f.copy()
        for _ in range(n):
            ref = ndi.uniform_filter(ref, size=(L3, L1), mode=mode)
        if boundary != kernels.SYMMETRIC and n > 1:
            # uniform_filter extends each pass's output again; a half-sample
            # symmetric extension commutes with a symmetric kernel, the zero
            # and replicate extensions do not, so compare those away from borders
            r = n * max(L1, L3)
            out, ref = out[r:-r or None, r:-r or None], ref[r:-r or None, r:-r or None]
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("boundary", [0, 1, 2])
def test_constant_image_preserved(boundary):
    H, W = 9, 12
    f = np.full((H, W), 7.0)
    cov = wl.random_cov_field(H, W, seed=1, sigma_range=(0.5, 4), rho_range=(1, 3))
    for n in (1, 2, 3):
        out = modular.filter_modular(f, cov, n, boundary, q=8, bits=64, out_dtype=np.float64,
                                     return_all=True)
        if boundary == kernels.ZERO:
            # interior pixels whose kernel stays inside the image
            Lf = out["L"]
            ok = np.ones((H, W), bool)
            for y in range(H):
                for x in range(W):
                    xm, xM, ym, yM = params.tap_extent(Lf[:, y, x], n)
                    ok[y, x] = (x + xm >= 0) and (x + xM < W) and (y + ym >= 0) and (y + yM < H)
            assert (out["out"][ok] == 7.0).all()
        else:
            assert (out["out"] == 7.0).all()


def _pure_python_running_sums(fe, n, mod):
    """Restricted running sums written as explicit loops over each line."""
    Hp, Wp = len(fe), len(fe[0])
    S = [[int(v) % mod for v in row] for row in fe]
    for (dx, dy) in (params.DIRS[0], params.DIRS[2], params.DIRS[1], params.DIRS[3]):
        for _ in range(n):
            T = [[0] * Wp for _ in range(Hp)]
            for y in range(Hp):
                for x in range(Wp):
                    acc, xx, yy = 0, x, y
                    while 0 <= xx < Wp and 0 <= yy < Hp:
                        acc += S[yy][xx]
                        xx, yy = xx - dx, yy - dy
                    T[y][x] = acc % mod
            S = T
    return S


@pytest.mark.parametrize("n", [1, 2])
def test_running_sums_equal_pure_python(n):
    rng = np.random.default_rng(7)
    fe = rng.integers(-2 ** 40, 2 ** 40, size=(6, 7)).astype(np.int64)
    S = modular.preintegrate(fe, n, 64)
    ref = _pure_python_running_sums(fe.tolist(), n, 1 << 64)
    assert S.tolist() == ref
    S128 = modular.preintegrate(fe, n, 128)
    ref128 = _pure_python_running_sums(fe.tolist(), n, 1 << 128)
    got = (S128.lo.astype(object) + (S128.hi.astype(object) << 64)).tolist()
    assert got == ref128


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
def test_modular_equals_direct_bit_exact(n, boundary):
    H, W = 14, 19
    f = wl.random_integer_image(H, W, seed=10 * n + boundary, lo=-500, hi=500)
    cov = wl.random_cov_field(H, W, seed=n, sigma_range=(0.3, 3.5), rho_range=(1, 4))
    for bits in (64, 128):
        r = modular.filter_modular(f, cov, n, boundary, q=3, bits=bits, out_dtype=np.float64,
                                   return_all=True)
        fq = quantize(f, 3)
        acc = kernels.correlate_exact(fq, r["L"], n, boundary)
        assert all(int(acc[y, x]) == int(r["acc"][y, x]) for y in range(H) for x in range(W))


def test_modular_wraparound_is_harmless():
    # q large enough that the running sums wrap mod 2^64 many times while every
    # accumulator still fits in 63 bits.
    H, W, n = 12, 12, 2
    f = wl.random_integer_image(H, W, seed=3, lo=0, hi=255)
    cov = wl.constant_cov_field(H, W, 2.0, 0.5, 1.5)
    r = modular.filter_modular(f, cov, n, 2, q=40, bits=64, out_dtype=np.float64, return_all=True)
    S = r["S"].view(np.int64)
    assert np.abs(S.astype(np.float64)).max() > 2.0 ** 60  # wrapped / large
    acc = kernels.correlate_exact(quantize(f, 40), r["L"], n, 2)
    assert all(int(acc[y, x]) == int(r["acc"][y, x]) for y in range(H) for x in range(W))
    # and 128-bit agrees
    r2 = modular.filter_modular(f, cov, n, 2, q=40, bits=128, out_dtype=np.float64, return_all=True)
    np.testing.assert_array_equal(r["out"], r2["out"])


def test_fixed_point_output_close_to_float64_definition():
    H, W, n = 16, 16, 2
    f = wl.blob_image(H, W, seed=0, n_blobs=5, sigma_range=(2, 5)).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=2, sigma_range=(0.5, 3), rho_range=(1, 3))
    out = modular.filter_modular(f, cov, n, 2, q=30, bits=64, out_dtype=np.float32, return_all=True)
    ref = kernels.correlate_f64(f.astype(np.float64), out["L"], n, 2)
    err = np.abs(out["out"].astype(np.float64) - ref).max()
    assert err <= 4 * 2.0 ** -24 * np.abs(ref).max() + 2.0 ** -30


def test_rn32_exact_rounding():
    from fractions import Fraction
    rng = np.random.default_rng(0)
    vals = [0, 1, -1, 2 ** 24 - 1, 2 ** 24 + 1, 2 ** 24 + 3, -(2 ** 25 + 2), 2 ** 62 + 2 ** 38,
            2 ** 62 + 2 ** 38 + 1, 2 ** 63 - 1, -(2 ** 63)]
    vals += [int(v) for v in rng.integers(-2 ** 63, 2 ** 63 - 1, size=500, dtype=np.int64)]
    for v in vals:
        r = rn_f32_int(v)
        # brute force: r must be a nearest float32 and ties must go to even
        a = float(r)
        up = float(np.nextafter(np.float32(a), np.float32(np.inf)))
        dn = float(np.nextafter(np.float32(a), np.float32(-np.inf)))
        e = abs(Fraction(a) - v)
        assert e <= abs(Fraction(up) - v) and e <= abs(Fraction(dn) - v)
        if e == abs(Fraction(up) - v) or e == abs(Fraction(dn) - v):
            assert int(np.float32(a).view(np.uint32)) % 2 == 0
    arr = np.array(vals, dtype=np.int64)
    np.testing.assert_array_equal(_rn32_array(arr), np.array([rn_f32_int(v) for v in vals]))


def test_finalize_small_exact():
    acc = np.array([[6, -9, 0]], dtype=np.int64)
    D = np.array([[3, 3, 7]], dtype=np.int64)
    np.testing.assert_array_equal(finalize(acc, D, 1, np.float64), [[1.0, -1.5, 0.0]])
    np.testing.assert_array_equal(finalize(acc, D, 1, np.float32), np.float32([[1.0, -1.5, 0.0]]))


def test_int64_kernel_equals_exact_kernel():
    rng = np.random.default_rng(11)
    for n in (1, 2, 3):
        for _ in range(5):
            L = tuple(int(v) for v in rng.integers(1, 9, size=4))
            if n % 2 == 1:
                L = tuple(2 * (v // 2) + 1 for v in L)
            K, ox, oy = kernels.kernel_d1(L, n)
            K2, ox2, oy2 = kernels.kernel_d1_int64(L, n)
            assert (ox, oy) == (ox2, oy2)
            np.testing.assert_array_equal(K.astype(np.int64), K2)


def test_sampled_exact_correlation_matches_full():
    H, W, n = 12, 15, 3
    f = wl.random_integer_image(H, W, seed=4, lo=0, hi=256)
    cov = wl.random_cov_field(H, W, seed=6, sigma_range=(0.5, 3), rho_range=(1, 3))
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    fq = quantize(f, 0)
    full = kernels.correlate_exact(fq, L, n, 2)
    pix = [(0, 0), (5, 7), (11, 14), (3, 12)]
    samp = kernels.correlate_exact_sampled(fq, L, n, 2, pix)
    for p in pix:
        assert samp[p] == full[p]
