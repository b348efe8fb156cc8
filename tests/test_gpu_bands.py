"""Row-band backward kernels on one GPU: each band's exact adjoint sums
(int64, or int128 for the continuous steps and 128-bit contexts) against
the oracle's adjoint of that band alone, and the bands assembled by the
library's halo add (the sums the add-exchange forms) and finalised against
the whole-image backward, bit for bit."""
import numpy as np
import pytest

import workloads as wl
from oracle import backward as ob
from oracle import modular, params
from tests.gpu_helpers import oracle_R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


@pytest.mark.parametrize("n,boundary,world", [(2, 2, 3), (1, 0, 2), (3, 1, 2), (2, 1, 4)])
def test_band_backward_assembles_to_whole_image(n, boundary, world):
    import torch
    from paper_1109_5114_gb300 import bands, bsf
    H, W = 150, 90
    gout = wl.uniform_image(H, W, seed=7, lo=-1.0, hi=1.0).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=8, sigma_range=(0.5, 3.0), rho_range=(1.0, 3.0))
    f = bsf.BoxSplineFilter(H, W, n, boundary, precision=1, frac_bits=10)
    tc = torch.from_numpy(cov).cuda()
    tg = torch.from_numpy(gout).cuda()
    f.plan(tc)
    R = oracle_R(cov, n, gpu=f.info().R)
    bands.check_bands(H, R, world)
    whole, _ = f.backward(tg, tc)
    qg = ob.grad_frac_bits(float(np.abs(gout).max()))   # the oracle's rule on max |gout| over the bands
    assert qg == bsf.bsf_grad_frac_bits(max(f.grad_absmax_rows(tg, *bands.band_bounds(H, world, r))
                                            for r in range(world)))
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    g = ob.quantize_weights(gout, modular.masses(L, n), qg)
    total = torch.zeros((H, W), dtype=torch.int64, device="cuda")
    for r in range(world):
        y0, y1 = bands.band_bounds(H, world, r)
        acc, a0, a1 = f.backward_rows(tg, tc, y0, y1, qg)
        g_band = np.zeros_like(g)
        g_band[y0:y1] = g[y0:y1]
        ref = ob.adjoint_modular_acc(g_band, L, n, boundary, R)
        np.testing.assert_array_equal(acc.cpu().numpy(), ref[a0:a1])
        f.grad_halo_add(total[a0:a1], acc)        # the library's modular add
    assembled = f.grad_finalize(total, qg)
    torch.cuda.synchronize()
    assert f.status() == 0
    np.testing.assert_array_equal(assembled.cpu().numpy(), whole.cpu().numpy())


def _to_pairs(acc_obj):
    """Python-integer sums as int128 two's complement (low, high) int64 pairs."""
    H, W = acc_obj.shape
    out = np.zeros((H, W, 2), dtype=np.uint64)
    m = (1 << 64) - 1
    for y in range(H):
        for x in range(W):
            v = int(acc_obj[y, x]) & ((1 << 128) - 1)
            out[y, x, 0] = v & m
            out[y, x, 1] = v >> 64
    return out.view(np.int64)


@pytest.mark.parametrize("prec,boundary,world", [(2, 2, 2), (1, 1, 2), (2, 0, 3)])
def test_band_backward_continuous_steps(prec, boundary, world):
    # continuous steps (128-bit adjoint sums, on 64- or 128-bit contexts):
    # each band's sums equal the oracle's adjoint of that band alone, and the
    # bands assembled by the library's halo add equal the whole-image backward
    import torch
    from oracle import continuous as cn
    from paper_1109_5114_gb300 import bands, bsf
    H, W, n = 66, 24, 2
    gout = wl.uniform_image(H, W, seed=17, lo=-1.0, hi=1.0).astype(np.float32)
    planes = wl.param_fields_logsig_theta_logrho(H, W, 18, logsig_range=(-1.0, 0.6), logrho_range=(0.0, 1.0))
    f = bsf.BoxSplineFilter(H, W, n, boundary, precision=prec, frac_bits=-1, step_rule=bsf.BSF_STEP_D2,
                            cov_kind=bsf.BSF_COV_LOGSIG_THETA_LOGRHO)
    tc = torch.from_numpy(planes).cuda()
    tg = torch.from_numpy(gout).cuda()
    f.plan(tc)
    R = oracle_R(planes, n, "d2", kind=1, gpu=f.info().R)
    bands.check_bands(H, R, world)
    assert f.info().grad_elem_bytes == 16
    whole, _ = f.backward(tg, tc, want_gimg=True, want_gcov=False)
    qg = cn.grad_frac_bits_d2(float(np.abs(gout).max()))
    assert qg == f.grad_frac_bits(max(f.grad_absmax_rows(tg, *bands.band_bounds(H, world, r))
                                      for r in range(world)))
    pix = [(y, x) for y in range(H) for x in range(W)]
    recs = cn.filter_d2_direct(np.zeros((H, W), dtype=np.int64), planes, n, boundary, pix, kind=1, R=R)
    total = torch.zeros((H, W, 2), dtype=torch.int64, device="cuda")
    for r in range(world):
        y0, y1 = bands.band_bounds(H, world, r)
        acc, a0, a1 = f.backward_rows(tg, tc, y0, y1, qg)
        gq = {p: cn.quantize_weight_d2(float(gout[p]), recs[p]["M"], qg) for p in pix if y0 <= p[0] < y1}
        ref = cn.adjoint_d2_acc(gq, planes, n, boundary, (H, W), kind=1, R=R)
        np.testing.assert_array_equal(acc.cpu().numpy(), _to_pairs(ref[a0:a1]))
        f.grad_halo_add(total[a0:a1], acc)
    assembled = f.grad_finalize(total, qg)
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    np.testing.assert_array_equal(assembled.cpu().numpy(), whole.cpu().numpy())


@pytest.mark.parametrize("n,world", [(2, 2), (3, 3)])
def test_band_backward_128bit_context(n, world):
    # integer steps on a 128-bit context: 128-bit band sums assemble to the
    # whole-image backward bit for bit
    import torch
    from paper_1109_5114_gb300 import bands, bsf
    H, W = 150, 70
    gout = wl.uniform_image(H, W, seed=21, lo=-1.0, hi=1.0).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=22, sigma_range=(0.5, 3.0), rho_range=(1.0, 3.0))
    f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=bsf.BSF_FIX128, frac_bits=30)
    tc, tg = torch.from_numpy(cov).cuda(), torch.from_numpy(gout).cuda()
    f.plan(tc)
    R = oracle_R(cov, n, gpu=f.info().R)
    bands.check_bands(H, R, world)
    whole, _ = f.backward(tg, tc)
    qg = ob.grad_frac_bits_wide(float(np.abs(gout).max()))
    assert qg == f.grad_frac_bits(float(np.abs(gout).max()))
    total = torch.zeros((H, W, 2), dtype=torch.int64, device="cuda")
    for r in range(world):
        y0, y1 = bands.band_bounds(H, world, r)
        acc, a0, a1 = f.backward_rows(tg, tc, y0, y1, qg)
        f.grad_halo_add(total[a0:a1], acc)
    assembled = f.grad_finalize(total, qg)
    torch.cuda.synchronize()
    assert f.status() == 0
    f.close()
    np.testing.assert_array_equal(assembled.cpu().numpy(), whole.cpu().numpy())
