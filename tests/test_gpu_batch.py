"""GPU parity of the batched form: images of uneven sizes, each with its own
covariance field, in one arena; every image bit-exact against the oracle in
the batched, graph-replayed and per-image modes."""
import numpy as np
import pytest

import workloads as wl
from oracle import config, modular, params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


@pytest.mark.parametrize("n", [1, 2])
def test_batch_bit_exact_all_modes(n):
    import torch
    from paper_1109_5114_gb300 import bsf
    sizes = wl.batch_sizes_loguniform(9, seed=3, lo=24, hi=300)
    imgs, covs = [], []
    for i, (H, W) in enumerate(sizes):
        imgs.append(wl.blob_image(H, W, seed=i, n_blobs=6, sigma_range=(2, 20)))
        covs.append(wl.random_cov_field(H, W, seed=50 + i, sigma_range=(0.5, 6.0), rho_range=(1.0, 3.0)))
    vmax = max(float(np.abs(im).max()) for im in imgs)
    bf = bsf.BatchFilter(n, "symmetric", frac_bits=-1, value_bound=vmax)
    d_imgs = [torch.from_numpy(a).cuda() for a in imgs]
    d_covs = [torch.from_numpy(c).cuda() for c in covs]
    d_outs = [torch.zeros(a.shape, dtype=torch.float32, device="cuda") for a in imgs]
    torch.cuda.synchronize()
    info = bf.plan(d_imgs, d_covs, d_outs, autotune=True)
    # one q for the batch: the automatic rule at the largest mass of any image
    mass = max(config.mass_bound(c, n) for c in covs)
    q = max(config.auto_frac_bits(vmax, mass, 64), 0)
    assert info.frac_bits == q
    refs = []
    for a, c in zip(imgs, covs):
        L, _ = params.integer_steps(c[0], c[1], c[2], n)
        R = max(int(params.reach(L, n).max()), 3 * n)
        refs.append(modular.filter_modular(a, c, n, 2, q=q, bits=64, out_dtype=np.float32, R=R))
    for flags in (0, bsf.BSF_BATCH_GRAPH, bsf.BSF_BATCH_GRAPH, bsf.BSF_BATCH_PER_IMAGE):
        for o in d_outs:
            o.fill_(float("nan"))
        torch.cuda.synchronize()
        bf.run(flags)
        assert bf.status() == 0
        for o, r in zip(d_outs, refs):
            np.testing.assert_array_equal(o.cpu().numpy(), r)
    assert bf.info().graph_ready == 1
    bf.close()
