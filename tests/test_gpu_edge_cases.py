"""Degenerate and extreme shapes for the later filter forms: the second
direction set and the pair, the sampled box spline, Algorithm 1, the 32-bit
running sums, the global passes against the fused tiles, and a zero field."""
import numpy as np
import pytest

import workloads as wl
from oracle import knight as kn
from oracle import modular, two_pass
from oracle import sampled as sp
from tests.gpu_helpers import oracle_R_two_pass, run_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 37), (29, 1), (2, 3), (5, 70)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


@pytest.mark.parametrize("shape", SHAPES)
def test_degenerate_shapes_second_set_pair_and_fix32(shape):
    H, W = shape
    img = wl.random_integer_image(H, W, seed=2, lo=0, hi=255).astype(np.uint8)
    cov = wl.constant_cov_field(H, W, 2.0, 0.9, 1.5)   # inside the second set's sector
    for n in (1, 2):
        g = run_gpu(img, cov, n, 2, q=6, directions=1)
        np.testing.assert_array_equal(g["out"], kn.filter_modular_k(img, cov, n, 2, q=6, R=g["R"]))
        g = run_gpu(img, cov, n, 2, q=6, directions=2)
        np.testing.assert_array_equal(g["out"], kn.algorithm2(img, cov, n, 2, q=6, R=g["R"])[0])
        for tiles_off in (False, True):
            g = run_gpu(img, cov, n, 1, q=0, precision=5, want_S=tiles_off)  # want_S turns the tiles off
            np.testing.assert_array_equal(g["out"], modular.filter_modular(img, cov, n, 1, q=0, bits=32, R=g["R"]))


@pytest.mark.parametrize("shape", SHAPES)
def test_degenerate_shapes_sampled_and_two_pass(shape):
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = shape
    img = wl.random_integer_image(H, W, seed=3, lo=-40, hi=40).astype(np.float32)
    cov = wl.constant_cov_field(H, W, 1.7, 0.4, 1.1)
    f = bsf.BoxSplineFilter(H, W, 1, "symmetric", frac_bits=12, step_rule=bsf.BSF_STEP_SAMPLED)
    out = f.filter(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda()).cpu().numpy()
    assert f.status() == 0
    f.close()
    np.testing.assert_array_equal(out, sp.filter_sampled(img, cov, 2, 12))
    f = bsf.BoxSplineFilter(H, W, 2, "replicate", frac_bits=16)
    out, s2 = f.filter_two_pass(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda(), want_sigma2=True)
    R = oracle_R_two_pass(cov, 2, gpu=f.info().R)
    assert f.status() == 0
    f.close()
    ref, s2_ref, _ = two_pass.algorithm1(img, cov, 2, 1, q=16, R=R)
    assert np.float32(s2) == s2_ref
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_zero_field_is_identity_in_every_form():
    # zero covariance: every box is one sample (or the shortest continuous
    # box), so the integer-step forms return the quantised image
    H, W = 19, 23
    img = wl.random_integer_image(H, W, seed=4, lo=-100, hi=100).astype(np.float32)
    cov = np.zeros((3, H, W), np.float32)
    for directions in (0, 1, 2):
        for n in (1, 2, 3):
            g = run_gpu(img, cov, n, 0, q=4, directions=directions)
            np.testing.assert_array_equal(g["out"], img)


def test_large_image_tiles_against_global_passes():
    # 4096 x 3000 with small kernels: the fused tiles and the global passes
    # agree bit for bit on the whole image (uint32 and uint64)
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 3000, 4096
    img = torch.from_numpy(wl.blob_image_u8(H, W, seed=5)).cuda()
    cov = torch.from_numpy(wl.diagonal_ramp_cov_field(H, W, sigma_hi=2.5, rho_hi=2.5)).cuda()
    for prec in (5, 1):
        outs = []
        for tiles in (1, 0):
            f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=prec, frac_bits=2)
            f.set_option(bsf.BSF_OPT_TILES, tiles)
            f.set_profiling(True)
            outs.append(f.filter(img, cov))
            prof = f.read_profile()
            assert f.status() == 0 and prof["tiles"][1] == tiles
            f.close()
        assert torch.equal(outs[0], outs[1])
