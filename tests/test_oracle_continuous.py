"""Pins of the continuous-step oracle (oracle/continuous.py) against closed
forms, the integer-step kernels, Proposition 1, finite differences and an
independent scale search.  CPU only."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import continuous as cn
from oracle import kernels, params
from workloads import synth

HS = list(range(512, 2600, 41)) + [1023, 1024, 1025, 1536, 2047, 2048, 2049, 512 * 7 + 3]


@pytest.mark.parametrize("n", [1, 2])
def test_line_kernel_matches_closed_form(n):
    # triangle of half-width lambda sampled at the integers (n = 2), cell
    # overlaps with the box of width lambda (n = 1), times 2^QW
    for Hh in HS:
        g, dg, j0, M, dM, ds = cn.line_data(Hh, n)
        r = Hh // 256 + 4
        for j in range(-r, r + 1):
            i = j - j0
            val = g[i] if 0 <= i < len(g) else 0
            assert val == cn.line_closed_form(Hh, n, j), (Hh, j)
        assert all(v >= 0 for v in g)
        val = lambda j: g[j - j0] if 0 <= j - j0 < len(g) else 0  # noqa: E731
        assert all(val(j) == val(-j) for j in range(r + 1))  # symmetric about 0


@pytest.mark.parametrize("n,Ls", [(1, (1, 3, 5, 9, 15)), (2, (1, 2, 3, 4, 7, 10))])
def test_admissible_integer_steps_reduce_to_d1(n, Ls):
    for L in Ls:
        g, _, j0, M, _, _ = cn.line_data(cn.HALF * L, n)
        nz = [i for i, v in enumerate(g) if v]
        core = g[nz[0]:nz[-1] + 1]
        assert tuple(v // cn.SCALE for v in core) == kernels.box_power_1d(L, n)
        assert all(v % cn.SCALE == 0 for v in core)
        assert j0 + nz[0] == -(n * (L - 1)) // 2
        assert M == cn.SCALE * L ** n
    # whole 2-D kernel
    for Lt in [(3, 5, 1, 3), (1, 1, 1, 1), (5, 3, 7, 1)]:
        K2, _, ox2, oy2, M2, *_ = cn.kernels_d2(tuple(cn.HALF * L for L in Lt), 1)
        K1, ox1, oy1 = kernels.kernel_d1(Lt, 1)
        nzy, nzx = np.nonzero(K2.astype(bool))
        sub = K2[nzy.min():nzy.max() + 1, nzx.min():nzx.max() + 1]
        assert sub.shape == K1.shape
        assert (sub == K1 * cn.SCALE ** 4).all()
        assert (ox2 - nzx.min(), oy2 - nzy.min()) == (ox1, oy1)
        assert M2 == kernels.kernel_mass(Lt, 1) * cn.SCALE ** 4


def test_mass_of_order_two_closed_form():
    # M = lambda^2 + (1/2) sum_t (-1)^t C(2,t) theta_t (1 - theta_t),
    # theta_t = frac(c - t lambda), c = lambda - 1
    for Hh in HS:
        lam = Fraction(Hh, cn.HALF)
        c = lam - 1
        s = Fraction(0)
        for t in range(3):
            qt = c - t * lam
            th = qt - math.floor(qt)
            s += (-1) ** t * math.comb(2, t) * th * (1 - th)
        M = cn.line_data(Hh, 2)[3]
        assert Fraction(M, cn.SCALE) == lam * lam + s / 2


def _closed_real(lam: Fraction, n: int, j: int) -> Fraction:
    if n == 2:
        return max(Fraction(0), lam - abs(j))
    return max(Fraction(0), min(Fraction(2 * j + 1, 2), lam / 2) - max(Fraction(2 * j - 1, 2), -lam / 2))


@pytest.mark.parametrize("n", [1, 2])
def test_derivative_kernel_is_right_derivative(n):
    eps = Fraction(1, 1 << 30)
    for Hh in HS:
        g, dg, j0, M, dM, ds = cn.line_data(Hh, n)
        lam = Fraction(Hh, cn.HALF)
        for i in range(-3, len(g) + 3):
            j = j0 + i
            d_exact = (_closed_real(lam + eps, n, j) - _closed_real(lam, n, j)) / eps
            val = dg[i] if 0 <= i < len(dg) else 0
            assert Fraction(val, cn.SCALE * ds) == d_exact, (Hh, j)
        assert dM == sum(dg)


def test_kernel_covariance_is_sum_of_line_variances():
    # Proposition 1: covariances of the four 1-D factors add, each along d_k
    for n, Hs in [(2, (700, 1300, 512, 2100)), (1, (1500, 600, 900, 1800))]:
        K, _, ox, oy, M, *_ = cn.kernels_d2(Hs, n)
        ys, xs = np.mgrid[0:K.shape[0], 0:K.shape[1]]
        X = xs - ox
        Y = ys - oy
        Kf = K
        tot = int(Kf.sum())
        assert tot == M
        mx = sum(int(v) * int(x) for v, x in zip(Kf.ravel(), X.ravel()))
        my = sum(int(v) * int(y) for v, y in zip(Kf.ravel(), Y.ravel()))
        assert mx == 0 and my == 0
        cxx = Fraction(sum(int(v) * int(x) ** 2 for v, x in zip(Kf.ravel(), X.ravel())), tot)
        cyy = Fraction(sum(int(v) * int(y) ** 2 for v, y in zip(Kf.ravel(), Y.ravel())), tot)
        cxy = Fraction(sum(int(v) * int(x) * int(y) for v, x, y in zip(Kf.ravel(), X.ravel(), Y.ravel())), tot)
        C = np.zeros((2, 2), dtype=object)
        C[:] = Fraction(0)
        for k, (dx, dy) in enumerate(params.DIRS):
            g, _, j0, Mk, _, _ = cn.line_data(Hs[k], n)
            var = Fraction(sum(v * (j0 + i) ** 2 for i, v in enumerate(g)), Mk)
            C[0, 0] += var * dx * dx
            C[0, 1] += var * dx * dy
            C[1, 1] += var * dy * dy
        assert (cxx, cxy, cyy) == (C[0, 0], C[0, 1], C[1, 1])
        # point symmetry about the origin: K(j) = K(-j)
        nzy, nzx = np.nonzero(K.astype(bool))
        assert all(K[2 * oy - y, 2 * ox - x] == K[y, x] for y, x in zip(nzy, nzx))


@pytest.mark.parametrize("n", [1, 2])
@pytest.mark.parametrize("bits", [64, 128])
def test_running_sum_pipeline_equals_definition(n, bits):
    H, W = 18, 15
    f = synth.random_integer_image(H, W, seed=11, lo=-60, hi=60)
    cov = synth.random_cov_field(H, W, seed=2, sigma_range=(0.5, 2.2), rho_range=(1.0, 3.0))
    for b in (kernels.ZERO, kernels.REPLICATE, kernels.SYMMETRIC):
        mod = cn.filter_d2_modular(f, cov, n, b, q=0, bits=bits)
        R = next(iter(mod.values()))["R"]
        dr = cn.filter_d2_direct(f.astype(np.int64), cov, n, b, list(mod), R=R)
        for p, a in mod.items():
            c = dr[p]
            assert (a["acc"], a["dacc"], a["M"], a["dMk"]) == (c["acc"], c["dacc"], c["M"], c["dMk"]), p


@pytest.mark.parametrize("n", [1, 2])
def test_constant_image_has_zero_jacobian(n):
    H, W = 16, 16
    f = np.full((H, W), 37, dtype=np.int64)
    fields = synth.param_fields_logsig_theta_logrho(H, W, seed=9, logsig_range=(0.0, 1.0))
    for b in (kernels.REPLICATE, kernels.SYMMETRIC):
        rec = cn.filter_d2_direct(f, fields, n, b, [(0, 0), (7, 9), (15, 3)], kind=1)
        for r in rec.values():
            assert r["acc"] == 37 * r["M"]
            assert all(Fraction(v) == 0 for v in cn.jacobian_steps(r, 0))


def test_identity_steps_out_of_reach():
    f = synth.random_integer_image(12, 12, seed=1)
    cov = synth.constant_cov_field(12, 12, 9.0, 0.0, 9.0)
    rec = cn.filter_d2_direct(f.astype(np.int64), cov, 2, kernels.SYMMETRIC, [(5, 6)], R=3)
    r = rec[(5, 6)]
    assert r["far"] and r["H"] == (cn.HALF,) * 4
    assert r["acc"] == int(f[5, 6]) * r["M"] and r["M"] == cn.SCALE ** 4


def test_float64_solve_matches_bruteforce_and_finite_differences():
    rng = np.random.default_rng(5)
    for _ in range(12):
        sig = rng.uniform(0.5, 8.0)
        rho = rng.uniform(1.0, 4.0)
        th = rng.uniform(0, math.pi)
        C = params.cov_from_sigma_rho_theta(sig, rho, th)
        for n in (1, 2):
            A = np.array([complex(a).real for a in cn.solve_scales_f64(*[float(c) for c in C], n)])
            Ab = params.solve_scales_bruteforce(*[float(c) for c in C], n, grid=4001)
            assert np.allclose(A, Ab, rtol=1e-6, atol=1e-6 * A.max())
            Jc = cn.dsteps_dplanes([float(c) for c in C], 0, n)
            h = 1e-6
            for j in range(3):
                pp = [float(c) for c in C]
                pm = list(pp)
                pp[j] += h
                pm[j] -= h
                fd = (np.real(cn.steps_f64(pp, 0, n)) - np.real(cn.steps_f64(pm, 0, n))) / (2 * h)
                assert np.allclose(Jc[:, j], fd, rtol=1e-5, atol=1e-7)


def test_float32_elementary_functions():
    x = np.linspace(-87, 88, 400001).astype(np.float32)
    e = cn.exp_f32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    assert (np.abs(e - ref) <= 1.5 * np.spacing(ref.astype(np.float32)).astype(np.float64)).all()
    x = np.linspace(-20, 20, 400001).astype(np.float32)
    s, c = cn.sincos_f32(x)
    assert np.abs(s - np.sin(x.astype(np.float64))).max() < 2.0 ** -23
    assert np.abs(c - np.cos(x.astype(np.float64))).max() < 2.0 ** -23
    # quadrant bookkeeping: sin^2 + cos^2 = 1, odd/even symmetry
    assert np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1).max() < 4e-7
    s2, c2 = cn.sincos_f32(-x)
    assert (s2 == -s).all() and (c2 == c).all()


def test_log_parameter_covariance():
    rng = np.random.default_rng(3)
    ls = rng.uniform(-1, 3, 500).astype(np.float32)
    th = rng.uniform(-0.2, math.pi + 0.2, 500).astype(np.float32)
    lr = rng.uniform(0, 1.1, 500).astype(np.float32)
    C = cn.cov_from_log_params(ls, th, lr)
    ref = params.cov_from_sigma_rho_theta(np.exp(ls.astype(np.float64)), np.exp(lr.astype(np.float64)),
                                          th.astype(np.float64))
    for a, b in zip(C, ref):
        scale = np.maximum(np.abs(ref[0]), np.abs(ref[2]))  # C12 is relative to the diagonal
        assert (np.abs(a - b) <= 4e-7 * scale).all()


@pytest.mark.parametrize("n", [1, 2])
def test_jacobian_matches_central_differences(n):
    # d out / d (log sigma, theta, log rho) against central differences (step
    # 1e-3) of the float64 filter with unquantised steps, at pixels whose
    # interpolation brackets do not change inside the difference interval
    H, W = 40, 40
    f = synth.blob_image(H, W, seed=0, n_blobs=12, sigma_range=(2.0, 6.0)).astype(np.float64)
    fields = synth.param_fields_logsig_theta_logrho(H, W, seed=4, logsig_range=(0.0, 1.2))
    q = 40
    pix = [(20, 20), (10, 30), (25, 12), (33, 33), (5, 5), (0, 39)]
    rec = cn.filter_d2_direct(cn.quantize(f, q, as_object=True), fields, n, kernels.SYMMETRIC, pix, kind=1)
    h = 1e-3
    checked = 0
    for (y, x) in pix:
        pl = fields[:, y, x].astype(np.float64)
        J = cn.jacobian_planes(rec[(y, x)], pl, 1, n, q)
        fd = np.zeros(3)
        kink = False
        for j in range(3):
            pp, pm = pl.copy(), pl.copy()
            pp[j] += h
            pm[j] -= h
            lp = np.real(cn.steps_f64(list(pp), 1, n))
            lm = np.real(cn.steps_f64(list(pm), 1, n))
            kink |= any(cn.brackets(a, n) != cn.brackets(b, n) for a, b in zip(lp, lm))
            fd[j] = (cn.filter_d2_f64_at(f, pp, 1, n, kernels.SYMMETRIC, y, x)
                     - cn.filter_d2_f64_at(f, pm, 1, n, kernels.SYMMETRIC, y, x)) / (2 * h)
        if kink:
            continue
        checked += 1
        assert np.allclose(J, fd, atol=0.02 * np.abs(fd).max() + 1e-6), ((y, x), J, fd)
    assert checked >= 4


def test_output_rule_and_orders_above_two_rejected():
    f = synth.uniform_image(10, 9, seed=2)
    cov = synth.constant_cov_field(10, 9, 2.0, 0.3, 1.5)
    q = 30
    rec = cn.filter_d2_modular(f, cov, 2, kernels.SYMMETRIC, q, bits=128, pixels=[(4, 4)])[(4, 4)]
    val = cn.output(rec, q, np.float64)
    exact = Fraction(rec["acc"], rec["M"] << q)
    assert abs(Fraction(float(val)) - exact) <= abs(exact) * Fraction(1, 1 << 50)
    with pytest.raises(ValueError):
        cn.line_taps(1024, 3)


@pytest.mark.parametrize("n", [1, 2])
def test_image_adjoint_identity(n):
    # <A f, g> = <f, A^T g> exactly, for integer f and integer weights g,
    # where A f is the definition's sum and A^T g the adjoint's
    H, W = 13, 11
    f = synth.random_integer_image(H, W, seed=2, lo=-20, hi=20).astype(np.int64)
    cov = synth.random_cov_field(H, W, seed=3, sigma_range=(0.4, 1.8), rho_range=(1.0, 3.0))
    rng = np.random.default_rng(n)
    for b in (kernels.ZERO, kernels.REPLICATE, kernels.SYMMETRIC):
        gq = {(y, x): int(rng.integers(-50, 50)) for y in range(H) for x in range(W)}
        fwd = cn.filter_d2_direct(f, cov, n, b, list(gq))
        lhs = sum(gq[p] * fwd[p]["acc"] for p in gq)
        adj = cn.adjoint_d2_acc(gq, cov, n, b, (H, W))
        rhs = sum(int(f[y, x]) * adj[y, x] for y in range(H) for x in range(W))
        assert lhs == rhs


def test_image_gradient_scale_rule():
    for m in (1e-30, 2.0 ** -7, 0.37, 0.5, 1.0, 3.0, 4.0, 1e6, 3e38):
        qg = cn.grad_frac_bits_d2(m)
        mf = float(np.float32(m))
        if 0 < qg < 126:
            assert 2.0 ** 117 < mf * 2.0 ** qg <= 2.0 ** 118
        assert 0 <= qg <= 126
    # weights: the float32 quotient, rounded half to even
    assert cn.quantize_weight_d2(1.5, 1, 0) == 2 and cn.quantize_weight_d2(2.5, 1, 0) == 2
    assert cn.quantize_weight_d2(-0.37, 2 ** 50, 100) == int(round(float(
        np.float32(np.float32(-0.37 * 2.0 ** 100) / np.float32(2.0 ** 50)))))
