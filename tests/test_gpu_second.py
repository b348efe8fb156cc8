"""GPU parity of the second direction set (Algorithm 3 with integer steps)
and of the pair switched by sector (Algorithm 2): steps, both sets of running
sums and the outputs bit for bit against oracle/knight.py."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import knight as kn
from oracle import params
from tests.gpu_helpers import oracle_S, oracle_S_second, run_gpu

pytestmark = pytest.mark.gpu

SECOND, PAIR = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _field(H, W, seed, smax=4.0, emax=6.0):
    """Covariances of every orientation and elongations up to emax (many
    beyond the first set's bound), trace 2 sigma^2 with sigma up to smax."""
    rng = np.random.default_rng(seed)
    s2 = rng.uniform(0.3, smax, (H, W)) ** 2
    e = rng.uniform(1.0, emax, (H, W))
    phi = rng.uniform(0, np.pi, (H, W))
    c, s = np.cos(phi), np.sin(phi)
    k = 2 * s2 / (1 + e)
    return np.stack([k * (e * c * c + s * s), k * (e - 1) * s * c, k * (e * s * s + c * c)]).astype(np.float32)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("rule", [0, 1])
def test_second_set_steps_bit_exact(n, rule):
    H, W = 37, 53
    cov = _field(H, W, seed=n + 10 * rule, smax=6.0, emax=12.0)
    img = np.zeros((H, W), np.float32)
    g = run_gpu(img, cov, n, 2, q=4, want_steps=True, step_rule=rule, directions=SECOND)
    L, fl = kn.integer_steps_k(cov[0], cov[1], cov[2], n, "paper" if rule else "corrected")
    np.testing.assert_array_equal(g["L"], L)
    assert g["info"].clamp_count == int(((fl & params.CLAMP_FLAG) != 0).sum())


@pytest.mark.parametrize("n", [1, 2, 3])
def test_pair_steps_and_sector_bit_exact(n):
    H, W = 41, 47
    cov = _field(H, W, seed=20 + n, emax=12.0)
    cov[:, 0, 0] = (2.0, 0.0, 2.0)      # isotropic: the first set
    cov[:, 0, 1] = (3.0, 1.0, 1.0)      # |C11 - C22| = 2 |C12|: inside the sector
    cov[:, 0, 2] = (4.0, 1.0, 1.0)      # |C11 - C22| = 3 |C12|: the boundary, first set
    img = np.zeros((H, W), np.float32)
    g = run_gpu(img, cov, n, 2, q=4, want_steps=True, directions=PAIR)
    mask, L, fl, _ = kn.pair_steps(cov, n)
    np.testing.assert_array_equal(g["second"], mask)
    np.testing.assert_array_equal(g["L"], L)
    assert not mask[0, 0] and mask[0, 1] and not mask[0, 2]
    assert g["info"].clamp_count == int(((fl & params.CLAMP_FLAG) != 0).sum())


@pytest.mark.parametrize("n,prec,shape", [(1, 1, (29, 70)), (2, 1, (150, 260)), (3, 1, (67, 131)),
                                          (1, 2, (88, 47)), (2, 2, (131, 140)), (3, 2, (40, 300))])
def test_second_set_running_sums_bit_exact(n, prec, shape):
    # padded heights above one 64-row chunk, odd and even row counts (the
    # row-parity grids of e2 and e3), widths across several 128-line blocks
    H, W = shape
    img = wl.random_integer_image(H, W, seed=n + W, lo=-300, hi=300).astype(np.float32)
    cov = _field(H, W, seed=n, smax=2.0, emax=3.0)
    g = run_gpu(img, cov, n, 2, q=5, precision=prec, want_S=True, directions=SECOND)
    bits = 64 if prec == 1 else 128
    S = oracle_S_second(img, n, 2, 5, g["R"], bits)
    if bits == 64:
        np.testing.assert_array_equal(g["S"], S)
    else:
        np.testing.assert_array_equal(g["S"][0], S.lo)
        np.testing.assert_array_equal(g["S"][1], S.hi)


def test_pair_holds_both_running_sums():
    H, W = 45, 66
    img = wl.random_integer_image(H, W, seed=3, lo=-100, hi=100).astype(np.float32)
    cov = _field(H, W, seed=4, smax=2.5)
    g = run_gpu(img, cov, 2, 1, q=6, want_S=True, directions=PAIR)
    np.testing.assert_array_equal(g["S"][0], oracle_S(img, 2, 1, 6, g["R"], 64))
    np.testing.assert_array_equal(g["S"][1], oracle_S_second(img, 2, 1, 6, g["R"], 64))


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_second_set_filter_bit_exact(n, boundary, dtype):
    H, W = 57, 83
    img = wl.blob_image(H, W, seed=n, n_blobs=6, sigma_range=(2, 8))
    img = (img * 255).clip(0, 255).astype(np.uint8) if dtype == np.uint8 else img.astype(np.float32)
    cov = _field(H, W, seed=30 + n, smax=3.0, emax=8.0)
    q = 20 if n < 3 else 12
    g = run_gpu(img, cov, n, boundary, q=q, directions=SECOND)
    ref = kn.filter_modular_k(img, cov, n, boundary, q=q, R=g["R"])
    np.testing.assert_array_equal(g["out"], ref)


@pytest.mark.parametrize("n,boundary,prec,out64", [(1, 2, 1, False), (2, 2, 1, False), (2, 0, 1, True),
                                                   (3, 1, 1, False), (2, 2, 2, False), (3, 2, 2, True)])
def test_pair_filter_bit_exact(n, boundary, prec, out64):
    H, W = 61, 77
    img = wl.blob_image(H, W, seed=40 + n, n_blobs=5, sigma_range=(2, 8)).astype(np.float32)
    cov = _field(H, W, seed=50 + n, smax=3.0, emax=9.0)
    q = 40 if prec == 2 else (20 if n < 3 else 12)
    odt = np.float64 if out64 else np.float32
    g = run_gpu(img, cov, n, boundary, q=q, precision=prec, out_dtype=odt, directions=PAIR)
    ref, mask, R = kn.algorithm2(img, cov, n, boundary, q=q, bits=64 if prec == 1 else 128, out_dtype=odt,
                                 R=g["R"])
    assert mask.any() and (~mask).any()
    np.testing.assert_array_equal(g["out"], ref)


def test_pair_clamps_less_than_either_set():
    H, W = 64, 64
    cov = _field(H, W, seed=60, smax=3.0, emax=9.0)
    img = np.zeros((H, W), np.float32)
    c = [run_gpu(img, cov, 2, 2, q=4, directions=d)["info"].clamp_count for d in (0, SECOND, PAIR)]
    assert c[2] < c[0] and c[2] < c[1]


@pytest.mark.parametrize("directions", [SECOND, PAIR])
def test_row_bands_equal_whole_image(directions):
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 70, 90
    img = torch.from_numpy(wl.blob_image(H, W, seed=7, n_blobs=5, sigma_range=(2, 8)).astype(np.float32)).cuda()
    cov = torch.from_numpy(_field(H, W, seed=8, smax=3.0)).cuda()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=20, directions=directions)
    whole = f.filter(img, cov).cpu().numpy()
    bands = [f.filter_rows(img, cov, y0, y1).cpu().numpy() for y0, y1 in ((0, 23), (23, 51), (51, 70))]
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    np.testing.assert_array_equal(np.concatenate(bands), whole)


def test_host_buffer_entry_with_the_pair():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 96, 112
    img = wl.blob_image(H, W, seed=9, n_blobs=5, sigma_range=(2, 8)).astype(np.float32)
    cov = _field(H, W, seed=10, smax=3.0)
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=20, directions=PAIR)
    dev = f.filter(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda()).cpu().numpy()
    h_out = torch.empty((H, W), dtype=torch.float32).pin_memory()
    for _ in range(3):   # eager, then graph capture, then replay
        f.filter_host(torch.from_numpy(img).pin_memory(), torch.from_numpy(cov).pin_memory(), h_out)
        np.testing.assert_array_equal(h_out.numpy(), dev)
    assert f.status() == 0
    f.close()


def test_second_set_argument_errors():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 16, 16
    img = torch.zeros((H, W), device="cuda")
    cov = torch.from_numpy(_field(H, W, seed=1)).cuda()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=8)
    with pytest.raises(bsf.BsfError):
        f.set_option(bsf.BSF_OPT_DIRECTIONS, 3)
    f.close()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=bsf.BSF_F64ACC, frac_bits=-1, directions=SECOND)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f.close()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=bsf.BSF_FIX128, frac_bits=8,
                            step_rule=bsf.BSF_STEP_D2, directions=PAIR)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f.close()
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", frac_bits=8, directions=PAIR)
    f.filter(img, cov)
    with pytest.raises(bsf.BsfError):
        f.backward(torch.ones((H, W), device="cuda"), cov)
    torch.cuda.synchronize()
    f.close()
