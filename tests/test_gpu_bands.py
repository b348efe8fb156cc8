"""Row-band backward kernels on one GPU: each band's exact int64 adjoint sums
against the oracle's adjoint of that band alone, and the bands assembled
(the sums the halo add-exchange forms) and finalised against the
whole-image backward, bit for bit."""
import numpy as np
import pytest

import workloads as wl
from oracle import backward as ob
from oracle import modular, params

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
    R = f.info().R
    bands.check_bands(H, R, world)
    whole, _ = f.backward(tg, tc)
    qg = bsf.bsf_grad_frac_bits(max(f.grad_absmax_rows(tg, *bands.band_bounds(H, world, r))
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
        total[a0:a1] += acc
    assembled = f.grad_finalize(total, qg)
    torch.cuda.synchronize()
    assert f.status() == 0
    np.testing.assert_array_equal(assembled.cpu().numpy(), whole.cpu().numpy())
