"""GPU parity of the 32-bit modular running sums (BSF_FIX32) and of the
automatic element width (BSF_FIX) against the oracle's modular pipelines
mod 2^32 / 2^64 / 2^128: running sums and outputs bit for bit."""
import numpy as np
import pytest

import workloads as wl
from oracle import knight as kn
from oracle import modular
from tests.gpu_helpers import oracle_S, oracle_S_second, run_gpu

pytestmark = pytest.mark.gpu

FIX, FIX32, FIX64, FIX128 = 0, 5, 1, 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _small_cov(H, W, seed):
    return wl.random_cov_field(H, W, seed=seed, sigma_range=(0.5, 1.8), rho_range=(1.0, 2.0))


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("directions", [0, 1])
def test_fix32_running_sums_bit_exact(n, directions):
    H, W = 77, 140   # two 64-row chunks, several 128-line blocks
    img = wl.random_integer_image(H, W, seed=n, lo=0, hi=255).astype(np.uint8)
    cov = _small_cov(H, W, n)
    g = run_gpu(img, cov, n, 2, q=0, precision=FIX32, want_S=True, directions=directions)
    assert g["info"].elem_bytes == 4
    ref = (oracle_S if directions == 0 else oracle_S_second)(img, n, 2, 0, g["R"], 32)
    np.testing.assert_array_equal(g["S"], ref)


@pytest.mark.parametrize("n,boundary", [(1, 0), (1, 2), (2, 1), (2, 2), (3, 2)])
@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_fix32_filter_bit_exact(n, boundary, dtype):
    H, W = 61, 90
    if dtype == np.uint8:
        img, q = wl.random_integer_image(H, W, seed=7, lo=0, hi=255).astype(np.uint8), 0
    else:
        img, q = wl.blob_image(H, W, seed=8, n_blobs=5, sigma_range=(2, 6)).astype(np.float32), 10
    cov = _small_cov(H, W, 10 + n)
    g = run_gpu(img, cov, n, boundary, q=q, precision=FIX32)
    assert g["status"] == 0
    ref = modular.filter_modular(img, cov, n, boundary, q=q, bits=32, R=g["R"])
    np.testing.assert_array_equal(g["out"], ref)
    # within the bound the 32-bit result is the 64-bit one
    np.testing.assert_array_equal(ref, modular.filter_modular(img, cov, n, boundary, q=q, bits=64, R=g["R"]))


@pytest.mark.parametrize("directions", [1, 2])
def test_fix32_second_set_and_pair(directions):
    H, W = 50, 73
    img = wl.random_integer_image(H, W, seed=4, lo=0, hi=255).astype(np.uint8)
    cov = _small_cov(H, W, 5)
    g = run_gpu(img, cov, 2, 2, q=0, precision=FIX32, directions=directions)
    if directions == 1:
        ref = kn.filter_modular_k(img, cov, 2, 2, q=0, bits=32, R=g["R"])
    else:
        ref, _, _ = kn.algorithm2(img, cov, 2, 2, q=0, bits=32, R=g["R"])
    np.testing.assert_array_equal(g["out"], ref)


def test_fix32_overflow_is_reported():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 40, 40
    img = torch.full((H, W), 255, dtype=torch.uint8, device="cuda")
    cov = torch.from_numpy(wl.random_cov_field(H, W, seed=1, sigma_range=(6, 8), rho_range=(1, 2))).cuda()
    f = bsf.BoxSplineFilter(H, W, 3, "symmetric", precision=FIX32, frac_bits=0)
    f.filter(img, cov)
    assert f.status() == bsf.BSF_EOVERFLOW
    f.close()


def test_automatic_width():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 64, 80
    img8 = wl.random_integer_image(H, W, seed=2, lo=0, hi=255).astype(np.uint8)
    # small kernels, uint8: 32 bits suffice at q = 0
    cov = _small_cov(H, W, 3)
    g = run_gpu(img8, cov, 2, 2, q=-1, precision=FIX)
    assert g["info"].elem_bytes == 4 and g["q"] >= 0
    np.testing.assert_array_equal(g["out"], modular.filter_modular(img8, cov, 2, 2, q=g["q"], bits=32, R=g["R"]))
    # float image: q must reach 25 - ceil(log2 max|f|) -> 64 bits
    imgf = wl.blob_image(H, W, seed=3, n_blobs=5, sigma_range=(2, 6)).astype(np.float32)
    g = run_gpu(imgf, cov, 2, 2, q=-1, precision=FIX)
    assert g["info"].elem_bytes == 8
    np.testing.assert_array_equal(g["out"], modular.filter_modular(imgf, cov, 2, 2, q=g["q"], bits=64, R=g["R"]))
    # a fixed q beyond 64 bits' reach -> 128 bits
    big = wl.random_cov_field(H, W, seed=4, sigma_range=(8, 10), rho_range=(1, 2))
    g = run_gpu(img8, big, 3, 2, q=40, precision=FIX)
    assert g["info"].elem_bytes == 16 and g["status"] == 0
    # the width follows each image: one context, small then large values
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=FIX, frac_bits=-1)
    tc = torch.from_numpy(cov).cuda()
    f.filter(torch.from_numpy(img8).cuda(), tc)
    torch.cuda.synchronize()
    e1 = f.info().elem_bytes
    f.filter(torch.from_numpy(imgf).cuda(), tc)
    torch.cuda.synchronize()
    e2 = f.info().elem_bytes
    assert (e1, e2) == (4, 8) and f.status() == 0
    f.close()


def test_fix32_argument_errors():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 16, 16
    cov = torch.from_numpy(_small_cov(H, W, 1)).cuda()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=FIX32, frac_bits=0, step_rule=bsf.BSF_STEP_D2)
    with pytest.raises(bsf.BsfError):
        f.filter(torch.zeros((H, W), device="cuda"), cov)
    f.close()
    with pytest.raises(bsf.BsfError):
        bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=FIX32, frac_bits=31)
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=FIX32, frac_bits=0)
    f.filter(torch.zeros((H, W), dtype=torch.uint8, device="cuda"), cov)
    # the backward reads no running sums: 64-bit adjoint sums on a 32-bit context
    g, _ = f.backward(torch.ones((H, W), device="cuda"), cov)
    torch.cuda.synchronize()
    assert f.status() == 0 and torch.isfinite(g).all()
    f.close()
