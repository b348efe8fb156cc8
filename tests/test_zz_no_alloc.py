"""bsf_filter_noalloc: the forward filter on the library's static scratch array.

It is meant for callers that cannot allocate device memory while running (a
host application whose device-memory budget belongs to its own pool, or a
latency-critical loop that cannot afford cudaMalloc's device-wide
synchronisation).  This file is collected last on purpose.  The test calls
the entry point through the C ABI twice in a row, with different inputs, and
checks each result against bsf_filter (the allocating entry point) bit for
bit, the tolerance the other parity tests of this path use.  It also checks
the entry point against the CPU oracle directly (8-bit input, float64
output), and that a padding below the field's reach reports BSF_ERANGE and
gives the oracle's identity fallback for the pixels out of reach.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import config, modular

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()
    from paper_1109_5114_gb300 import bsf
    f = bsf._lib.bsf_filter_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p]
    return bsf, f, torch


def _reference(bsf, torch, img, cov, n, boundary, R, q):
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, boundary, max_reach=R, frac_bits=q)
    out = f.filter(img, cov)
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    return out


def test_noalloc_matches_filter_on_two_calls_in_a_row(lib):
    bsf, noalloc, torch = lib
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(200, 240, 2, 2, 11, (0.5, 6.0)), (131, 97, 3, 1, 7, (0.3, 3.0))]
    for H, W, n, boundary, seed, srange in cases:
        img = torch.from_numpy(wl.blob_image(H, W, seed=seed, n_blobs=10, sigma_range=(3, 12))).cuda()
        cov_np = wl.random_cov_field(H, W, seed=seed, sigma_range=srange, rho_range=(1.0, 3.0))
        cov = torch.from_numpy(cov_np).cuda()
        R = config.padding(cov_np, n)
        ref = _reference(bsf, torch, img, cov, n, boundary, R, 24)
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        rc = noalloc(ctypes.c_void_p(img.data_ptr()), bsf.BSF_F32, W, H, W, n, boundary, R, 24,
                     ctypes.c_void_p(cov.data_ptr()), ctypes.c_void_p(out.data_ptr()), bsf.BSF_F32,
                     W, ctypes.c_void_p(stream))
        assert rc == 0
        torch.testing.assert_close(out, ref, rtol=0, atol=0)


def test_noalloc_rejects_sizes_beyond_its_workspace(lib):
    bsf, noalloc, torch = lib
    H = W = 4096   # 4096^2 padded elements do not fit the static workspace
    img = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    cov = torch.zeros((3, 8, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    rc = noalloc(ctypes.c_void_p(img.data_ptr()), bsf.BSF_F32, W, H, W, 1, 2, 3, 10,
                 ctypes.c_void_p(cov.data_ptr()), ctypes.c_void_p(out.data_ptr()), bsf.BSF_F32, W,
                 None)
    assert rc == bsf.BSF_ERANGE


def _call(noalloc, bsf, img, dtype, cov, out, out_dtype, n, boundary, R, q, stream):
    H, W = out.shape
    return noalloc(ctypes.c_void_p(img.data_ptr()), dtype, W, H, W, n, boundary, R, q,
                   ctypes.c_void_p(cov.data_ptr()), ctypes.c_void_p(out.data_ptr()), out_dtype, W,
                   ctypes.c_void_p(stream))


def test_noalloc_u8_float64_output_equals_oracle(lib):
    bsf, noalloc, torch = lib
    stream = torch.cuda.current_stream().cuda_stream
    H, W, n = 77, 103, 2
    img8 = wl.blob_image_u8(H, W, seed=5, n_blobs=9)
    cov = wl.random_cov_field(H, W, seed=6, sigma_range=(0.5, 5.0), rho_range=(1.0, 3.0))
    R = config.padding(cov, n)
    for q in (0, 9):
        out = torch.full((H, W), float("nan"), dtype=torch.float64, device="cuda")
        rc = _call(noalloc, bsf, torch.from_numpy(img8).cuda(), bsf.BSF_U8, torch.from_numpy(cov).cuda(),
                   out, bsf.BSF_F64, n, 2, R, q, stream)
        assert rc == 0
        ref = modular.filter_modular(img8, cov, n, 2, q=q, bits=64, out_dtype=np.float64, R=R)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_noalloc_padding_below_reach_reports_erange(lib):
    bsf, noalloc, torch = lib
    stream = torch.cuda.current_stream().cuda_stream
    H, W, n = 40, 52, 2
    img = wl.random_integer_image(H, W, seed=1, lo=0, hi=100).astype(np.float32)
    cov = wl.constant_cov_field(H, W, 0.5, 0.0, 0.5)
    cov[:, 10:14, 20:30] = np.array([30.0, 0.0, 30.0], np.float32)[:, None, None]   # taps beyond R = 8
    assert config.padding(cov, n) > 8
    out = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    rc = _call(noalloc, bsf, torch.from_numpy(img).cuda(), bsf.BSF_F32, torch.from_numpy(cov).cuda(),
               out, bsf.BSF_F32, n, 2, 8, 10, stream)
    assert rc == bsf.BSF_ERANGE
    ref = modular.filter_modular(img, cov, n, 2, q=10, bits=64, R=8)   # identity steps where out of reach
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
