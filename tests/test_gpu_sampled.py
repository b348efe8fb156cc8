"""GPU parity of the sampled continuous box spline (BSF_STEP_SAMPLED): the
running sums interpolated at continuous taps by the grid box spline, bit for
bit against oracle/sampled.py, which computes sum_m f(m) beta_a(p + tau - m)
with beta_a by exact polygon areas."""
import numpy as np
import pytest

import workloads as wl
from oracle import sampled as sp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _run(img, cov, boundary, q, precision=1, out64=False, directions=0):
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, 1, boundary, precision=precision, frac_bits=q,
                            step_rule=bsf.BSF_STEP_SAMPLED, directions=directions)
    out = f.filter(torch.from_numpy(np.ascontiguousarray(img)).cuda(), torch.from_numpy(cov).cuda(),
                   out_dtype=torch.float64 if out64 else torch.float32)
    torch.cuda.synchronize()
    st = f.status()
    info = f.info()
    f.close()
    return out.cpu().numpy(), st, info


@pytest.mark.parametrize("boundary,precision,out64", [(0, 1, False), (1, 1, False), (2, 1, True),
                                                      (2, 2, False), (0, 2, True)])
def test_sampled_bit_exact_small(boundary, precision, out64):
    H, W = 17, 20
    img = wl.blob_image(H, W, seed=boundary, n_blobs=4, sigma_range=(2, 6)).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=10 + boundary, sigma_range=(0.5, 2.5), rho_range=(1.0, 3.0))
    q = 8 if precision == 1 else 30
    got, st, info = _run(img, cov, boundary, q, precision, out64)
    assert st == 0
    ref = sp.filter_sampled(img, cov, boundary, q, out_dtype=np.float64 if out64 else np.float32)
    np.testing.assert_array_equal(got, ref)


def test_sampled_bit_exact_sampled_pixels_larger():
    # several 32 x 8 blocks, ragged; pixels on every border and inside
    H, W = 141, 203
    img = wl.random_integer_image(H, W, seed=3, lo=0, hi=255).astype(np.uint8)
    cov = wl.random_cov_field(H, W, seed=4, sigma_range=(0.8, 4.0), rho_range=(1.0, 3.5))
    got, st, info = _run(img, cov, 2, 4)
    assert st == 0
    rng = np.random.default_rng(5)
    pix = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0), (70, 0), (0, 101)]
    pix += [(int(rng.integers(H)), int(rng.integers(W))) for _ in range(40)]
    ref = sp.filter_sampled(img, cov, 2, 4, pixels=pix)
    for p in pix:
        assert got[p] == ref[p], p


def test_sampled_constant_image():
    H, W = 32, 40
    img = np.full((H, W), 7.0, np.float32)
    cov = wl.random_cov_field(H, W, seed=6, sigma_range=(1.0, 3.0), rho_range=(1.0, 2.0))
    got, st, info = _run(img, cov, 1, 10)
    assert st == 0
    # the sampled box spline's mass is sum_m beta_a(p + tau - m), close to 1
    assert np.abs(got - 7.0).max() < 0.3
    pix = [(0, 0), (5, 7), (31, 39)]
    ref = sp.filter_sampled(img, cov, 1, 10, pixels=pix)
    assert all(got[p] == ref[p] for p in pix)


def test_sampled_argument_errors():
    import torch

    from paper_1109_5114_gb300 import bsf
    with pytest.raises(bsf.BsfError):
        bsf.BoxSplineFilter(16, 16, 2, "symmetric", frac_bits=8, step_rule=bsf.BSF_STEP_SAMPLED)
    cov = torch.from_numpy(wl.random_cov_field(16, 16, seed=1, sigma_range=(1, 2), rho_range=(1, 2))).cuda()
    img = torch.zeros((16, 16), device="cuda")
    f = bsf.BoxSplineFilter(16, 16, 1, "symmetric", precision=bsf.BSF_FIX32, frac_bits=0,
                            step_rule=bsf.BSF_STEP_SAMPLED)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f.close()
    f = bsf.BoxSplineFilter(16, 16, 1, "symmetric", frac_bits=8, step_rule=bsf.BSF_STEP_SAMPLED)
    f.filter(img, cov)
    with pytest.raises(bsf.BsfError):
        f.backward(torch.ones((16, 16), device="cuda"), cov)
    torch.cuda.synchronize()
    f.close()
    f = bsf.BoxSplineFilter(16, 16, 1, "symmetric", precision=bsf.BSF_FIX128, frac_bits=8,
                            step_rule=bsf.BSF_STEP_D2, directions=bsf.BSF_DIRS_PAIR)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f.close()


@pytest.mark.parametrize("directions,boundary,precision,out64", [(1, 2, 1, False), (1, 0, 2, True),
                                                                 (2, 2, 1, False), (2, 1, 2, False)])
def test_sampled_second_set_and_pair_bit_exact(directions, boundary, precision, out64):
    # Algorithm 3 as printed (beta'_a through the running sums of the second
    # set interpolated by beta'_b) and Algorithm 2 with both sampled box
    # splines, against the exact-rational definitions
    H, W = 15, 18
    img = wl.blob_image(H, W, seed=directions + boundary, n_blobs=4, sigma_range=(2, 6)).astype(np.float32)
    rng = np.random.default_rng(30 + directions)
    phi = rng.uniform(0, np.pi, (H, W))
    e = rng.uniform(1.0, 4.0, (H, W))
    s2 = rng.uniform(0.8, 3.0, (H, W))
    c, sn = np.cos(phi), np.sin(phi)
    k = 2 * s2 / (1 + e)
    cov = np.stack([k * (e * c * c + sn * sn), k * (e - 1) * sn * c, k * (e * sn * sn + c * c)]).astype(np.float32)
    q = 8 if precision == 1 else 30
    odt = np.float64 if out64 else np.float32
    got, st, info = _run(img, cov, boundary, q, precision, out64, directions=directions)
    assert st == 0
    if directions == 1:
        ref = sp.filter_sampled_k(img, cov, boundary, q, out_dtype=odt)
    else:
        ref = sp.filter_sampled_pair(img, cov, boundary, q, out_dtype=odt)
    np.testing.assert_array_equal(got, ref)
