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
