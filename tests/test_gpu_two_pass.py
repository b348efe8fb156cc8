"""GPU parity of Algorithm 1 (isotropic pass, then the residual pass).

bsf_filter_two_pass against oracle.two_pass.algorithm1 on the same seeded
inputs: sigma^2 equal as float32, the output bit for bit (both passes are the
fixed-point pipeline with one explicit q).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import continuous as cn
from oracle import two_pass
from tests.gpu_helpers import oracle_R_two_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _run(img, cov, n, boundary, q, precision=1, frac=0.5, cov_kind=0, out64=False):
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, boundary, precision=precision, frac_bits=q, cov_kind=cov_kind)
    out = torch.empty((H, W), dtype=torch.float64 if out64 else torch.float32, device="cuda")
    out, s2 = f.filter_two_pass(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda(), frac,
                                out=out, want_sigma2=True)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = oracle_R_two_pass(cov, n, frac, cov_kind, gpu=f.info().R)
    f.close()
    return out.cpu().numpy(), np.float32(s2), R


@pytest.mark.parametrize("n,boundary,precision", [(1, 0, 1), (1, 2, 1), (2, 1, 1), (2, 2, 1),
                                                  (2, 0, 2), (3, 2, 2)])
def test_two_pass_bit_exact(n, boundary, precision):
    H, W = 83, 150   # several stencil tiles, ragged in both directions
    img = wl.blob_image(H, W, seed=20 + n, n_blobs=7, sigma_range=(2, 9))
    cov = wl.random_cov_field(H, W, seed=30 + boundary, sigma_range=(0.8, 3.5), rho_range=(1.0, 3.0))
    got, s2, R = _run(img, cov, n, boundary, q=18 if precision == 1 else 40, precision=precision)
    ref, s2_ref, _ = two_pass.algorithm1(img, cov, n, boundary, q=18 if precision == 1 else 40, R=R,
                                         bits=64 if precision == 1 else 128)
    assert s2 == s2_ref and s2 > 0
    np.testing.assert_array_equal(got, ref)


def test_two_pass_float64_output_and_fraction():
    H, W = 40, 57
    img = wl.random_integer_image(H, W, seed=3, lo=0, hi=255).astype(np.uint8)
    cov = wl.random_cov_field(H, W, seed=4, sigma_range=(1.0, 3.0), rho_range=(1.0, 2.5))
    got, s2, R = _run(img, cov, 2, 2, q=20, frac=0.3, out64=True)
    ref, s2_ref, _ = two_pass.algorithm1(img, cov, 2, 2, q=20, R=R, frac=0.3, out_dtype=np.float64)
    assert s2 == s2_ref
    np.testing.assert_array_equal(got, ref)


def test_two_pass_log_parameter_field():
    from paper_1109_5114_gb300 import bsf
    H, W = 35, 44
    rng = np.random.default_rng(5)
    planes = np.stack([rng.uniform(-0.3, 1.0, (H, W)), rng.uniform(-np.pi, np.pi, (H, W)),
                       rng.uniform(0.0, 1.0, (H, W))]).astype(np.float32)
    img = wl.blob_image(H, W, seed=6, n_blobs=4, sigma_range=(2, 6))
    got, s2, R = _run(img, planes, 2, 2, q=18, cov_kind=bsf.BSF_COV_LOGSIG_THETA_LOGRHO)
    C = np.stack(cn.cov_from_log_params(planes[0], planes[1], planes[2]))
    ref, s2_ref, _ = two_pass.algorithm1(img, C, 2, 2, q=18, R=R)
    assert s2 == s2_ref
    np.testing.assert_array_equal(got, ref)


def test_zero_bound_reduces_to_one_pass():
    # an axis-aligned pixel with a vanishing variance has bound 0, so
    # sigma^2 = 0: the isotropic pass is the identity on an integer image and
    # the two-pass result is the one-pass filter of the field
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 30, 41
    img = wl.random_integer_image(H, W, seed=8, lo=-100, hi=100).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=9, sigma_range=(1.0, 3.0), rho_range=(1.0, 2.0))
    cov[:, 7, 9] = (0.0, 0.0, 2.0)
    got, s2, R = _run(img, cov, 2, 2, q=16)
    assert s2 == 0.0
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=16, max_reach=R)
    one = f.filter(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda()).cpu().numpy()
    f.close()
    np.testing.assert_array_equal(got, one)


def test_two_pass_argument_errors():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 16, 16
    img = torch.zeros((H, W), device="cuda")
    cov = torch.from_numpy(wl.random_cov_field(H, W, seed=1, sigma_range=(1, 2), rho_range=(1, 2))).cuda()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=16)
    for frac in (0.0, 1.0, -0.5, float("nan")):
        with pytest.raises(bsf.BsfError):
            f.filter_two_pass(img, cov, frac)
    f.close()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=bsf.BSF_FIX128, frac_bits=16,
                            step_rule=bsf.BSF_STEP_D2)
    with pytest.raises(bsf.BsfError):
        f.filter_two_pass(img, cov)
    f.close()


@pytest.mark.parametrize("case", ["mixed", "constant", "near_isotropic"])
def test_sigma2_exact_on_hard_fields(case):
    # the device finds the minimum through a float32 interval per pixel and
    # evaluates the float64 bound only where the minimum can lie; sigma^2
    # must still equal the oracle's on fields where many intervals overlap
    H, W = 64, 96
    rng = np.random.default_rng(11)
    if case == "constant":
        cov = np.empty((3, H, W), np.float32)
        cov[0], cov[1], cov[2] = 2.5, 0.7, 1.25
    elif case == "near_isotropic":
        c = rng.uniform(1.0, 1.0 + 1e-6, (H, W))
        cov = np.stack([c, rng.uniform(-1e-7, 1e-7, (H, W)), c * (1 + 1e-7)]).astype(np.float32)
    else:
        s = rng.uniform(0.05, 300.0, (H, W))
        r = rng.choice([1.0, 1.0 + 1e-6, 1.5, 2.5], (H, W))
        th = rng.choice([0.0, 1e-20, np.pi / 4, rng.uniform(-np.pi, np.pi)], (H, W))
        k = 2 * s / (1 + r)
        c, sn = np.cos(th), np.sin(th)
        cov = np.stack([k * (r * c * c + sn * sn), k * (r - 1) * sn * c, k * (r * sn * sn + c * c)]).astype(np.float32)
    img = wl.random_integer_image(H, W, seed=2, lo=0, hi=200).astype(np.float32)
    got, s2, R = _run(img, cov, 1, 2, q=16)
    assert s2 == two_pass.sigma2_global(cov)
    ref, _, _ = two_pass.algorithm1(img, cov, 1, 2, q=16, R=R)
    np.testing.assert_array_equal(got, ref)
