"""GPU parity of the backward pass (image gradient) against the oracle's adjoint."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import backward, params
from tests.gpu_helpers import oracle_R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _gpu_backward(img, cov, gout, n, boundary, mode=0):
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, boundary, frac_bits=20)
    f.set_option(bsf.BSF_OPT_SCAN_MODE, mode)
    tc = torch.from_numpy(cov).cuda()
    f.filter(torch.from_numpy(img).cuda(), tc)
    gimg, gcov = f.backward(torch.from_numpy(gout).cuda(), tc, want_gcov=True)
    torch.cuda.synchronize()
    st = f.status()
    R = f.info().R
    f.close()
    return gimg.cpu().numpy(), gcov.cpu().numpy(), st, R


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
def test_backward_bit_exact_vs_oracle_adjoint(n, boundary):
    H, W = 37, 52
    rng = np.random.default_rng(3 * n + boundary)
    img = wl.blob_image(H, W, seed=n, n_blobs=5).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=20 + n, sigma_range=(0.3, 4.0), rho_range=(1.0, 3.0))
    gout = rng.normal(size=(H, W)).astype(np.float32)
    g, gc, st, R = _gpu_backward(img, cov, gout, n, boundary)
    assert st == 0
    R = oracle_R(cov, n, gpu=R)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    qg = backward.grad_frac_bits(np.abs(gout).max())
    ref = backward.adjoint_modular(gout, L, n, boundary, qg, R)
    np.testing.assert_array_equal(g, ref)
    assert (gc == 0).all()


def test_backward_matches_exact_adjoint_and_scan_modes():
    H, W, n = 64, 80, 2
    rng = np.random.default_rng(9)
    img = wl.blob_image(H, W, seed=4, n_blobs=6).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=5, sigma_range=(0.5, 6.0), rho_range=(1.0, 3.5))
    gout = rng.normal(size=(H, W)).astype(np.float32)
    g0, _, st0, _ = _gpu_backward(img, cov, gout, n, 2, mode=0)
    g1, _, st1, _ = _gpu_backward(img, cov, gout, n, 2, mode=1)
    assert st0 == 0 and st1 == 0
    np.testing.assert_array_equal(g0, g1)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    exact = backward.adjoint_f64(gout.astype(np.float64), L, n, 2)
    np.testing.assert_allclose(g0, exact, rtol=1e-5, atol=1e-5 * np.abs(exact).max())


def test_autograd_gradient_through_the_library():
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W, n = 40, 33, 2
    img = torch.from_numpy(wl.blob_image(H, W, seed=1, n_blobs=4)).cuda().requires_grad_(True)
    cov = torch.from_numpy(wl.random_cov_field(H, W, seed=2, sigma_range=(0.5, 3.0),
                                               rho_range=(1.0, 2.0))).cuda()
    f = bsf.BoxSplineFilter(H, W, n, "symmetric", frac_bits=24)
    out = bsf.box_spline_filter(img, cov, f)
    w = torch.linspace(-1, 1, H * W, device="cuda").reshape(H, W)
    loss = (out * w).sum()
    loss.backward()
    g_ref, _ = f.backward(w.contiguous(), cov)
    torch.cuda.synchronize()
    assert f.status() == 0
    torch.testing.assert_close(img.grad, g_ref, rtol=0, atol=0)
    f.close()


@pytest.mark.parametrize("n,boundary", [(1, 2), (2, 0), (3, 1)])
def test_backward_on_128bit_context_bit_exact(n, boundary):
    # a context with uint128 running sums takes the 128-bit adjoint format
    # (qg = 118 - ceil(log2 max|gout|)); bit-exact against the oracle's
    # definition in that format
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = 23, 31
    rng = np.random.default_rng(40 + n)
    img = wl.blob_image(H, W, seed=n, n_blobs=5).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=41 + n, sigma_range=(0.3, 4.0), rho_range=(1.0, 3.0))
    gout = rng.normal(size=(H, W)).astype(np.float32)
    f = bsf.BoxSplineFilter(H, W, n, boundary, precision=bsf.BSF_FIX128, frac_bits=40)
    tc = torch.from_numpy(cov).cuda()
    f.filter(torch.from_numpy(img).cuda(), tc)
    assert f.info().grad_elem_bytes == 16
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tc)
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    np.testing.assert_array_equal(gimg.cpu().numpy(), backward.adjoint_direct_wide(gout, L, n, boundary))


def test_backward_on_128bit_context_large_kernels():
    # masses near 2^64 (n = 3, steps ~ 40): the 128-bit format stays within
    # float32 accuracy of the exact adjoint, bit-exact against the oracle
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W, n = 9, 11, 3
    rng = np.random.default_rng(3)
    img8 = wl.random_integer_image(H, W, seed=4, lo=0, hi=255).astype(np.uint8)
    cov = wl.random_cov_field(H, W, seed=12, sigma_range=(24.0, 28.0), rho_range=(1.0, 2.0))
    gout = rng.normal(size=(H, W)).astype(np.float32)
    f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=bsf.BSF_FIX128, frac_bits=0)
    tc = torch.from_numpy(cov).cuda()
    f.filter(torch.from_numpy(img8).cuda(), tc)
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tc)
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    got = gimg.cpu().numpy()
    np.testing.assert_array_equal(got, backward.adjoint_direct_wide(gout, L, n, 2))
    exact = backward.adjoint_f64(gout.astype(np.float64), L, n, 2)
    np.testing.assert_allclose(got, exact, rtol=2e-6, atol=2e-6 * np.abs(exact).max())


def test_backward_equal_on_32_and_64_bit_contexts():
    # the backward reads no running sums: a context whose forward took 32-bit
    # sums gives the 64-bit context's gradient bit for bit
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W, n = 40, 57, 2
    img8 = wl.random_integer_image(H, W, seed=6, lo=0, hi=255).astype(np.uint8)
    cov = wl.random_cov_field(H, W, seed=7, sigma_range=(0.5, 1.6), rho_range=(1.0, 2.0))
    gout = torch.from_numpy(np.random.default_rng(8).normal(size=(H, W)).astype(np.float32)).cuda()
    tc = torch.from_numpy(cov).cuda()
    outs = []
    for prec in (bsf.BSF_FIX32, bsf.BSF_FIX64):
        f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=prec, frac_bits=0)
        f.filter(torch.from_numpy(img8).cuda(), tc)
        assert f.info().elem_bytes == (4 if prec == bsf.BSF_FIX32 else 8) and f.info().grad_elem_bytes == 8
        g, _ = f.backward(gout, tc)
        torch.cuda.synchronize()
        assert f.status() == 0
        outs.append(g.cpu().numpy())
        f.close()
    np.testing.assert_array_equal(outs[0], outs[1])
