"""GPU parity of the fused tile filter (tile-restarted pre-integration and
the stencil in one kernel, BSF_OPT_TILES): bit for bit against the oracle's
modular pipeline and against the global passes, and the accuracy the
restarted float64 sums keep."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import kernels, modular, params
from tests.gpu_helpers import oracle_R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _run(img, cov, n, boundary, q, precision=1, tiles=1, out64=False, rows=None):
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, boundary, precision=precision, frac_bits=q)
    f.set_option(bsf.BSF_OPT_TILES, tiles)
    f.set_profiling(True)
    ti = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    tc = torch.from_numpy(cov).cuda()
    odt = torch.float64 if out64 else torch.float32
    if rows is None:
        out = f.filter(ti, tc, out_dtype=odt)
    else:
        out = torch.cat([f.filter_rows(ti, tc, y0, y1, out=torch.empty((y1 - y0, W), dtype=odt, device="cuda"))
                         for y0, y1 in rows])
    prof = f.read_profile()
    st = f.status()
    info = f.info()
    f.close()
    return out.cpu().numpy(), info, st, prof


def _cov(H, W, seed, smax=2.5):
    return wl.random_cov_field(H, W, seed=seed, sigma_range=(0.5, smax), rho_range=(1.0, 3.0))


@pytest.mark.parametrize("n,boundary", list(itertools.product([1, 2, 3], [0, 1, 2])))
@pytest.mark.parametrize("dtype", [np.uint8, np.float32, np.float64])
def test_tiles_bit_exact_vs_oracle(n, boundary, dtype):
    H, W = 150, 211   # ragged in both directions against 64 / 96 / 128 tiles
    if dtype == np.uint8:
        img = wl.random_integer_image(H, W, seed=n, lo=0, hi=255).astype(np.uint8)
    else:
        img = wl.blob_image(H, W, seed=n + boundary, n_blobs=8, sigma_range=(2, 9)).astype(dtype)
    cov = _cov(H, W, seed=10 * n + boundary)
    q = 16 if n < 3 else 10
    out, info, st, prof = _run(img, cov, n, boundary, q)
    assert st == 0 and prof["tiles"][1] == 1 and prof["rows"][1] == 0
    ref = modular.filter_modular(img, cov, n, boundary, q=q, R=oracle_R(cov, n, gpu=info.R))
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("precision,n", [(5, 1), (5, 2), (2, 2), (2, 3), (1, 3)])
def test_tiles_precisions_equal_global_passes(precision, n):
    H, W = 97, 260
    img = wl.random_integer_image(H, W, seed=5, lo=0, hi=255).astype(np.uint8)
    cov = _cov(H, W, seed=6, smax=1.8 if precision == 5 else 3.0)
    q = 0 if precision == 5 else 24
    a, info, st_a, pa = _run(img, cov, n, 2, q, precision=precision, tiles=1, out64=True)
    b, _, st_b, pb = _run(img, cov, n, 2, q, precision=precision, tiles=0, out64=True)
    assert st_a == st_b == 0 and pa["tiles"][1] == 1 and pb["tiles"][1] == 0
    np.testing.assert_array_equal(a, b)
    bits = {5: 32, 1: 64, 2: 128}[precision]
    np.testing.assert_array_equal(a, modular.filter_modular(img, cov, n, 2, q=q, bits=bits, R=oracle_R(cov, n, gpu=info.R),
                                                            out_dtype=np.float64))


def test_tiny_image_and_bands():
    img = wl.blob_image(40, 33, seed=1, n_blobs=3, sigma_range=(2, 5)).astype(np.float32)
    cov = _cov(40, 33, seed=2)
    out, info, st, prof = _run(img, cov, 2, 2, 18)
    assert prof["tiles"][1] == 1
    np.testing.assert_array_equal(out, modular.filter_modular(img, cov, 2, 2, q=18, R=oracle_R(cov, 2, gpu=info.R)))
    H, W = 200, 150
    img = wl.blob_image(H, W, seed=3, n_blobs=6, sigma_range=(2, 8)).astype(np.float32)
    cov = _cov(H, W, seed=4)
    whole, info, _, _ = _run(img, cov, 2, 1, 18)
    bands, _, st, prof = _run(img, cov, 2, 1, 18, rows=[(0, 70), (70, 71), (71, 200)])
    assert st == 0 and prof["tiles"][1] == 3
    np.testing.assert_array_equal(bands, whole)


def test_large_padding_takes_the_global_passes():
    H, W = 96, 96
    img = wl.blob_image(H, W, seed=5, n_blobs=4, sigma_range=(2, 8)).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=6, sigma_range=(20, 26), rho_range=(1, 2))
    out, info, st, prof = _run(img, cov, 2, 2, 12)
    assert info.R > 60 and prof["tiles"][1] == 0 and prof["rows"][1] == 1
    np.testing.assert_array_equal(out, modular.filter_modular(img, cov, 2, 2, q=12, R=oracle_R(cov, 2, gpu=info.R)))


@pytest.mark.parametrize("n,bound,precision", [(1, 1e-8, 3), (2, 1e-3, 3), (1, 1e-5, 4)])
def test_restarted_float_sums_stay_accurate(n, bound, precision):
    # float64 (precision 3) or compensated float32 (precision 4) running
    # sums over a whole 1024^2 image lose most digits for n = 2; restarted per
    # tile they are bounded by the window (P ~ 90):
    # about P^(4n) / 2^(2n) max|f|, whose float64 rounding, over (n+1)^4 taps
    # with weights up to 2^(4(n-1)), is ~1e-11 (n = 1) and ~1e-5 (n = 2) of
    # the mass
    H = W = 1024
    img = wl.blob_image(H, W, seed=7).astype(np.float32)
    cov = _cov(H, W, seed=8, smax=2.0)
    exact, info, _, _ = _run(img, cov, n, 2, 30, precision=1, out64=True)
    tiled, _, st, prof = _run(img, cov, n, 2, -1, precision=precision, tiles=1, out64=True)
    glob, _, _, _ = _run(img, cov, n, 2, -1, precision=precision, tiles=0, out64=True)
    assert prof["tiles"][1] == 1
    scale = np.abs(exact).max()
    e_tiled = np.abs(tiled - exact).max() / scale
    e_glob = np.abs(glob - exact).max() / scale
    assert e_tiled < bound
    assert e_glob > 100 * e_tiled


def test_overflow_in_a_tile_is_reported():
    import torch

    from paper_1109_5114_gb300 import bsf
    H, W = 64, 64
    img = torch.full((H, W), 255, dtype=torch.uint8, device="cuda")
    cov = torch.from_numpy(wl.random_cov_field(H, W, seed=1, sigma_range=(4, 5), rho_range=(1, 2))).cuda()
    f = bsf.BoxSplineFilter(H, W, 3, "symmetric", precision=5, frac_bits=0)
    f.set_profiling(True)
    f.filter(img, cov)
    assert f.read_profile()["tiles"][1] == 1
    assert f.status() == bsf.BSF_EOVERFLOW
    f.close()


@pytest.mark.parametrize("directions,n,precision", [(1, 1, 1), (1, 2, 1), (1, 3, 2), (2, 1, 1), (2, 2, 1),
                                                    (2, 2, 5), (2, 3, 1)])
def test_tiles_of_the_second_set_and_the_pair(directions, n, precision):
    # the fused tiles with the second direction set (its running sums walked
    # along (2,1), (1,2), (-1,2), (-2,1) in the window) and with the pair
    # (two windows per block): equal to the global passes and to the oracle
    import torch

    from oracle import knight as kn
    from paper_1109_5114_gb300 import bsf
    H, W = 131, 170
    img = wl.random_integer_image(H, W, seed=n + 10 * directions, lo=0, hi=255).astype(np.uint8)
    cov = _cov(H, W, seed=20 + n, smax=1.6 if precision == 5 else 2.2)
    q = 0 if precision == 5 else 8
    outs, profs, R = [], [], None
    for tiles in (1, 0):
        f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=precision, frac_bits=q, directions=directions)
        f.set_option(bsf.BSF_OPT_TILES, tiles)
        f.set_profiling(True)
        out = f.filter(torch.from_numpy(img).cuda(), torch.from_numpy(cov).cuda())
        profs.append(f.read_profile())
        assert f.status() == 0
        R = oracle_R(cov, n, dirs="second" if directions == 1 else "pair", gpu=f.info().R)
        outs.append(out.cpu().numpy())
        f.close()
    assert profs[0]["tiles"][1] == 1 and profs[1]["tiles"][1] == 0
    np.testing.assert_array_equal(outs[0], outs[1])
    bits = {5: 32, 1: 64, 2: 128}[precision]
    if directions == 1:
        ref = kn.filter_modular_k(img, cov, n, 2, q=q, bits=bits, R=R)
    else:
        ref = kn.algorithm2(img, cov, n, 2, q=q, bits=bits, R=R)[0]
    np.testing.assert_array_equal(outs[0], ref)
