"""bsf_filter_noalloc: the forward filter on the library's static scratch array.

It is meant for callers that cannot allocate device memory while running (a
host application whose device-memory budget belongs to its own pool, or a
latency-critical loop that cannot afford cudaMalloc's device-wide
synchronisation).  This file is collected last on purpose.  The test calls
the entry point through the C ABI twice in a row, with different inputs, and
checks each result against bsf_filter (the allocating entry point) bit for
bit, the tolerance the other parity tests of this path use.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

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
        cov = torch.from_numpy(wl.random_cov_field(H, W, seed=seed, sigma_range=srange,
                                                   rho_range=(1.0, 3.0))).cuda()
        ref_f = bsf.BoxSplineFilter(H, W, n, boundary, frac_bits=24)
        R = ref_f.plan(cov).R
        ref_f.close()
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
