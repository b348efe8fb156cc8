"""GPU parity at the full sizes of the benchmarked workloads, in the launch
configuration bench.py times (bsf_filter through the C ABI, automatic or fixed
q as stated).

* 256^2 float64 uniform image, n = 1, C = 16 I, symmetric, float64 output,
  q = 40: bit-exact against the modular oracle on the whole image, and within
  1e-12 relative of the unquantised float64 definition.
* 2048^2 float32 blob image, n = 2, the space-variant ramp field, symmetric,
  automatic q, float32 output (the bench workload): bit-exact against the
  modular oracle on the whole image; sampled pixels within 1e-5 relative of
  the float64 definition.
* 8192^2 uint8 blob image, n = 3, smooth random field (sigma 2-32 px, rho 1-3),
  uint128 running sums, q = 0: sampled pixels bit-exact against the exact
  direct correlation.
* The image gradients of the two benchmarked backward passes: the 2048^2
  workload (integer steps, 64-bit adjoint sums) on the whole image against
  the oracle's transposed pipeline, and one 1024^2 image of the
  differentiation workload (continuous steps, 128-bit adjoint sums, the
  shared-memory window scatter) with gout nonzero on two windows (one at a
  corner, where the extension folds, one inside) against the oracle's direct
  adjoint of those pixels' kernels.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kernels, modular, params
from oracle.rounding import finalize, quantize
from tests.gpu_helpers import oracle_R, oracle_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _gpu(img, cov, n, q, precision, out_dtype, value_bound=None):
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=precision, frac_bits=q,
                            value_bound=value_bound)
    tc = torch.from_numpy(cov).cuda()
    f.plan(tc)
    out = f.filter(torch.from_numpy(img).cuda(), tc,
                   out_dtype=torch.float64 if out_dtype == np.float64 else torch.float32)
    torch.cuda.synchronize()
    st = f.status()
    info = f.info()
    res = out.cpu().numpy()
    f.close()
    return res, st, info


def _sample_pixels(H, W, k, seed):
    rng = np.random.default_rng(seed)
    pix = {(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0), (H // 2, W // 2)}
    while len(pix) < k:
        pix.add((int(rng.integers(0, H)), int(rng.integers(0, W))))
    return sorted(pix)


def test_tiny_256_float64_bit_exact():
    H = W = 256
    img = wl.uniform_image(H, W, seed=0)
    cov = wl.constant_cov_field(H, W, 16.0, 0.0, 16.0)
    out, st, info = _gpu(img, cov, 1, 40, 1, np.float64)
    assert st == 0 and info.R == 13 == oracle_R(cov, 1)
    ref = modular.filter_modular(img, cov, 1, 2, q=40, bits=64, out_dtype=np.float64, R=13)
    np.testing.assert_array_equal(out, ref)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], 1)
    pix = _sample_pixels(H, W, 64, 1)
    exact = kernels.correlate_f64(img, L, 1, 2, pixels=pix)
    for p in pix:
        assert abs(out[p] - exact[p]) <= 1e-12 * abs(exact[p])


def test_spacevariant_2048_bit_exact_whole_image():
    H = W = 2048
    img = wl.blob_image(H, W, seed=0)
    cov = wl.diagonal_ramp_cov_field(H, W)
    vmax = float(np.abs(img).max())
    out, st, info = _gpu(img, cov, 2, -1, 1, np.float32, value_bound=vmax)
    assert st == 0
    R = oracle_R(cov, 2, gpu=info.R)
    _, q = oracle_q(img, cov, 2, -1, 64, gpu=info.frac_bits, vmax=vmax)
    ref = modular.filter_modular(img, cov, 2, 2, q=q, bits=64, out_dtype=np.float32, R=R)
    np.testing.assert_array_equal(out, ref)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], 2)
    pix = _sample_pixels(H, W, 24, 2)
    exact = kernels.correlate_f64(img.astype(np.float64), L, 2, 2, pixels=pix)
    scale = float(np.abs(ref).max())
    for p in pix:
        assert abs(float(out[p]) - exact[p]) <= 1e-5 * max(abs(exact[p]), 1e-3 * scale)


def test_spacevariant_2048_backward_bit_exact_whole_image():
    """The forward + backward configuration of the benchmark (automatic q,
    64-bit context, f.backward): the image gradient of a seeded gout, every
    pixel bit-exact against the oracle's transposed running-sum pipeline."""
    import torch
    from oracle import backward
    from paper_1109_5114_gb300 import bsf
    H = W = 2048
    img = wl.blob_image(H, W, seed=0)
    cov = wl.diagonal_ramp_cov_field(H, W)
    gout = wl.uniform_image(H, W, seed=77, lo=-1, hi=1).astype(np.float32)
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=1, frac_bits=-1,
                            value_bound=float(np.abs(img).max()))
    tc = torch.from_numpy(cov).cuda()
    f.plan(tc)
    f.filter(torch.from_numpy(img).cuda(), tc)
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tc)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = oracle_R(cov, 2, gpu=f.info().R)
    got = gimg.cpu().numpy()
    f.close()
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], 2)
    qg = backward.grad_frac_bits(float(np.abs(gout).max()))
    np.testing.assert_array_equal(got, backward.adjoint_modular(gout, L, 2, kernels.SYMMETRIC, qg, R))


def test_differentiation_image_gradient_full_size_windows():
    """One 1024^2 image of the differentiation workload (the bench's context:
    uint128, continuous steps, log-parameter fields): gout nonzero on a
    12 x 24 window at the top-left corner and one inside, zero elsewhere, so
    that the oracle's direct adjoint stays affordable while the scatter runs
    over the whole image with the workload's fields; every pixel of the
    image gradient bit-exact."""
    import math
    import torch
    import bench
    from oracle import continuous as cn
    from oracle.rounding import rn_f32_int
    from paper_1109_5114_gb300 import bsf
    side = 1024
    imgs, fields, _ = bench.diff_inputs(1, side)
    fl = fields[0]
    u = wl.uniform_image(side, side, seed=78, lo=-1, hi=1).astype(np.float32)
    gout = np.zeros((side, side), np.float32)
    for win in ((slice(0, 12), slice(0, 24)), (slice(500, 512), slice(600, 624))):
        gout[win] = u[win]
    f = bsf.BoxSplineFilter(side, side, 2, "symmetric", precision=bsf.BSF_FIX128, frac_bits=-1,
                            value_bound=float(np.abs(imgs[0]).max()), step_rule=bsf.BSF_STEP_D2,
                            cov_kind=bsf.BSF_COV_LOGSIG_THETA_LOGRHO)
    tf = torch.from_numpy(fl).cuda()
    f.plan(tf)
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tf, want_gimg=True, want_gcov=False)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = oracle_R(fl, 2, "d2", kind=1, gpu=f.info().R)
    got = gimg.cpu().numpy()
    f.close()
    qg = cn.grad_frac_bits_d2(float(np.abs(gout).max()))
    gq = {}
    for y, x in zip(*np.nonzero(gout)):
        Hs = cn._pixel_steps(fl, 1, 2, int(y), int(x), R)[0]
        M = math.prod(cn.line_data(h, 2)[3] for h in Hs)  # the mass of the pixel's kernel
        gq[(int(y), int(x))] = cn.quantize_weight_d2(float(gout[y, x]), M, qg)
    acc = cn.adjoint_d2_acc(gq, fl, 2, kernels.SYMMETRIC, (side, side), kind=1, R=R)
    ref = np.zeros((side, side), np.float32)
    for y, x in zip(*np.nonzero(acc != 0)):
        ref[y, x] = np.float32(rn_f32_int(acc[y, x]) * np.float32(2.0 ** -qg))
    np.testing.assert_array_equal(got, ref)


def test_precision_8192_u8_uint128_sampled_bit_exact():
    H = W = 8192
    img = wl.blob_image_u8(H, W, seed=0)
    cov = wl.random_cov_field(H, W, seed=0, sigma_range=(2.0, 32.0), rho_range=(1.0, 3.0))
    out, st, info = _gpu(img, cov, 3, 0, 2, np.float32)
    assert st == 0
    n = 3
    pix = _sample_pixels(H, W, 48, 3)
    ys = np.array([p[0] for p in pix])
    xs = np.array([p[1] for p in pix])
    sub = cov[:, ys, xs][:, :, None]
    L = params.integer_steps(sub[0], sub[1], sub[2], n)[0][:, :, 0]
    Lfield = np.zeros((4, H, W), dtype=np.int64)
    Lfield[:, ys, xs] = L
    keep = [p for i, p in enumerate(pix) if kernels.kernel_mass(L[:, i], n) < (1 << 62)]
    acc = kernels.correlate_exact_sampled(quantize(img, 0), Lfield, n, 2, keep)
    for p in keep:
        D = np.array([kernels.kernel_mass(Lfield[:, p[0], p[1]], n)], dtype=object)
        ref = finalize(np.array([acc[p]], dtype=object), D, 0, np.float32)[0]
        assert out[p] == ref, p
    assert len(keep) >= 40


def test_differentiation_workload_one_image_full_size():
    """One 1024^2 image of the differentiation workload (blob seed 0, smooth
    log sigma / theta / log rho fields), continuous steps n = 2, uint128,
    automatic q, float32 output with the Jacobian (the call bench.py times):
    sampled outputs bit-exact against the oracle's running-sum pipeline on
    the whole padded image; the Jacobian within the tolerance of
    test_gpu_continuous at the same pixels; and against central differences
    (step 1e-3, float64, unquantised steps) of the float64 definition."""
    import torch
    import bench
    from oracle import continuous as cn
    from paper_1109_5114_gb300 import bsf
    imgs, fields, _ = bench.diff_inputs(1, 1024)
    img, fl = imgs[0], fields[0]
    side = 1024
    f = bsf.BoxSplineFilter(side, side, 2, "symmetric", precision=bsf.BSF_FIX128, frac_bits=-1,
                            value_bound=float(np.abs(img).max()), step_rule=bsf.BSF_STEP_D2,
                            cov_kind=bsf.BSF_COV_LOGSIG_THETA_LOGRHO)
    tf = torch.from_numpy(fl).cuda()
    f.plan(tf)
    out, J = f.filter_jacobian(torch.from_numpy(img).cuda(), tf)
    torch.cuda.synchronize()
    assert f.status() == 0
    info = f.info()
    R = oracle_R(fl, 2, "d2", kind=1, gpu=info.R)
    _, q = oracle_q(img, fl, 2, -1, 128, "d2", kind=1, gpu=info.frac_bits, vmax=float(np.abs(img).max()))
    out, J = out.cpu().numpy(), J.cpu().numpy()
    rng = np.random.default_rng(0)
    pix = sorted({(int(y), int(x)) for y, x in zip(rng.integers(0, side, 256), rng.integers(0, side, 256))}
                 | {(0, 0), (side - 1, side - 1), (0, side - 1), (side - 1, 0)})
    rec = cn.filter_d2_modular(img, fl, 2, kernels.SYMMETRIC, q, bits=128, kind=1,
                               R=R, pixels=pix)
    assert not any(r["far"] for r in rec.values())
    ref = np.array([cn.output(rec[p], q) for p in pix], dtype=np.float32)
    np.testing.assert_array_equal(np.array([out[p] for p in pix]), ref)
    refJ = np.array([cn.jacobian_planes(rec[p], fl[:, p[0], p[1]].astype(np.float64), 1, 2,
                                        q) for p in pix])
    gotJ = np.array([J[:, p[0], p[1]] for p in pix])
    for c in range(3):
        scale = np.abs(refJ[:, c]).max()
        assert (np.abs(gotJ[:, c] - refJ[:, c]) <= 2e-4 * scale + 1e-3 * np.abs(refJ[:, c])).all()
    # central differences of the unquantised float64 filter
    h = 1e-3
    checked = 0
    for (y, x) in pix[:12]:
        pl = fl[:, y, x].astype(np.float64)
        fd = np.zeros(3)
        kink = False
        for j in range(3):
            pp, pm = pl.copy(), pl.copy()
            pp[j] += h
            pm[j] -= h
            lp = np.real(cn.steps_f64(list(pp), 1, 2))
            lm = np.real(cn.steps_f64(list(pm), 1, 2))
            kink |= any(cn.brackets(a, 2) != cn.brackets(b, 2) for a, b in zip(lp, lm))
            fd[j] = (cn.filter_d2_f64_at(img, pp, 1, 2, kernels.SYMMETRIC, y, x)
                     - cn.filter_d2_f64_at(img, pm, 1, 2, kernels.SYMMETRIC, y, x)) / (2 * h)
        if kink:
            continue
        checked += 1
        assert np.allclose(J[:, y, x], fd, atol=0.02 * np.abs(fd).max() + 1e-6), ((y, x), J[:, y, x], fd)
    assert checked >= 6
