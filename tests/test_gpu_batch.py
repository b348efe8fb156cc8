"""GPU parity of the batched form: images of uneven sizes, each with its own
covariance field, in one arena; every image bit-exact against the oracle in
the batched, graph-replayed, per-image and persistent (one launch, direct and
graph-replayed) modes, for every work-item shape of the persistent launch;
the persistent launch's bounded waits run out when a phase never signals,
and the batch works normally afterwards."""
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
    P = bsf.BSF_BATCH_PERSISTENT
    for flags in (0, bsf.BSF_BATCH_GRAPH, bsf.BSF_BATCH_GRAPH, bsf.BSF_BATCH_PER_IMAGE, P,
                  P | bsf.BSF_BATCH_GRAPH, P | bsf.BSF_BATCH_GRAPH):
        for o in d_outs:
            o.fill_(float("nan"))
        torch.cuda.synchronize()
        bf.run(flags)
        assert bf.status() == 0
        for o, r in zip(d_outs, refs):
            np.testing.assert_array_equal(o.cpu().numpy(), r)
    info = bf.info()
    assert info.graph_ready == 1 and info.persist_graph_ready == 1
    assert info.persist_items > 0 and info.persist_grid > 0
    bf.close()


def test_batch64_full_size_persistent_graph_sampled_images():
    """The benchmark's batch (64 images, sides log-uniform in [128, 2048],
    seed 1; sigma 1-24 px; n = 2), planned with the autotuner and run as the
    bench's headline mode (one persistent launch replayed from a CUDA graph):
    the largest image, the smallest and six seeded others bit-exact on the
    whole image against the oracle (the batch's one q, each image's R)."""
    import torch
    from paper_1109_5114_gb300 import bsf
    sizes = wl.batch_sizes_loguniform(64, seed=1, lo=128, hi=2048)
    imgs, covs = [], []
    for i, (h, w) in enumerate(sizes):
        imgs.append(wl.blob_image(h, w, seed=1000 + i))
        covs.append(wl.random_cov_field(h, w, seed=2000 + 3 * i, sigma_range=(1.0, 24.0), rho_range=(1.0, 3.0)))
    vmax = max(float(np.abs(a).max()) for a in imgs)
    d_imgs = [torch.from_numpy(a).cuda() for a in imgs]
    d_covs = [torch.from_numpy(c).cuda() for c in covs]
    d_outs = [torch.full(a.shape, float("nan"), dtype=torch.float32, device="cuda") for a in imgs]
    bf = bsf.BatchFilter(2, "symmetric", frac_bits=-1, value_bound=vmax)
    torch.cuda.synchronize()
    info = bf.plan(d_imgs, d_covs, d_outs, autotune=True)
    mass = max(config.mass_bound(c, 2) for c in covs)
    q = max(config.auto_frac_bits(vmax, mass, 64), 0)
    assert info.frac_bits == q
    bf.run(bsf.BSF_BATCH_PERSISTENT | bsf.BSF_BATCH_GRAPH)
    bf.run(bsf.BSF_BATCH_PERSISTENT | bsf.BSF_BATCH_GRAPH)
    assert bf.status() == 0
    px = np.array([h * w for h, w in sizes])
    rng = np.random.default_rng(9)
    pick = {int(px.argmax()), int(px.argmin())} | {int(i) for i in rng.choice(64, 6, replace=False)}
    for i in sorted(pick):
        ref = modular.filter_modular(imgs[i], covs[i], 2, 2, q=q, bits=64, out_dtype=np.float32,
                                     R=config.padding(covs[i], 2))
        np.testing.assert_array_equal(d_outs[i].cpu().numpy(), ref)
    bf.close()


def _small_batch(n, seed0=0, count=7):
    import torch
    sizes = wl.batch_sizes_loguniform(count, seed=5 + seed0, lo=20, hi=260)
    imgs, covs = [], []
    for i, (H, W) in enumerate(sizes):
        imgs.append(wl.blob_image(H, W, seed=seed0 + i, n_blobs=6, sigma_range=(2, 20)))
        covs.append(wl.random_cov_field(H, W, seed=70 + seed0 + i, sigma_range=(0.5, 5.0), rho_range=(1.0, 3.0)))
    vmax = max(float(np.abs(im).max()) for im in imgs)
    refs_q = None
    d_imgs = [torch.from_numpy(a).cuda() for a in imgs]
    d_covs = [torch.from_numpy(c).cuda() for c in covs]
    d_outs = [torch.zeros(a.shape, dtype=torch.float32, device="cuda") for a in imgs]
    return imgs, covs, vmax, refs_q, d_imgs, d_covs, d_outs


def _refs(imgs, covs, n, q):
    return [modular.filter_modular(a, c, n, 2, q=q, bits=64, out_dtype=np.float32, R=config.padding(c, n))
            for a, c in zip(imgs, covs)]


@pytest.mark.parametrize("n", [1, 2, 3])
def test_persistent_shapes_bit_exact(n):
    # every work-item shape and block count of the persistent launch gives
    # the oracle's outputs (the tuner may pick any of them)
    import torch
    from paper_1109_5114_gb300 import bsf
    imgs, covs, vmax, _, d_imgs, d_covs, d_outs = _small_batch(n, seed0=10 * n)
    bf = bsf.BatchFilter(n, "symmetric", frac_bits=-1, value_bound=vmax)
    info = bf.plan(d_imgs, d_covs, d_outs)
    refs = _refs(imgs, covs, n, info.frac_bits)
    for rows, tile_rows, per_sm, group_mb in ((1, 8, 0, 0), (8, 16, 1, 1), (3, 32, 2, 2), (64, 64, 0, 48)):
        bf.set_option(bsf.BSF_BATCH_OPT_ROWS_PER_ITEM, rows)
        bf.set_option(bsf.BSF_BATCH_OPT_STENCIL_ROWS, tile_rows)
        bf.set_option(bsf.BSF_BATCH_OPT_BLOCKS_PER_SM, per_sm)
        bf.set_option(bsf.BSF_BATCH_OPT_GROUP_MB, group_mb)   # 1 MiB: about one image per group
        for o in d_outs:
            o.fill_(float("nan"))
        bf.run(bsf.BSF_BATCH_PERSISTENT)
        assert bf.status() == 0
        inf = bf.info()
        assert (inf.rows_per_item, inf.stencil_tile_rows) == (rows, tile_rows)
        assert inf.persist_groups >= 1 and (group_mb != 0 or inf.persist_groups == 1)
        for o, r in zip(d_outs, refs):
            np.testing.assert_array_equal(o.cpu().numpy(), r)
    bf.close()


def test_persistent_wait_times_out_and_batch_stays_usable():
    # failure injection: image 0's row phase never signals, so every item
    # waiting on it runs out of polls; the launch must end with BSF_ETIMEOUT
    # (no hang, no fault) and the batch must work normally afterwards
    from paper_1109_5114_gb300 import bsf
    imgs, covs, vmax, _, d_imgs, d_covs, d_outs = _small_batch(2, seed0=3, count=5)
    bf = bsf.BatchFilter(2, "symmetric", frac_bits=-1, value_bound=vmax)
    info = bf.plan(d_imgs, d_covs, d_outs)
    bf.set_option(bsf.BSF_BATCH_OPT_WAIT_LIMIT, 2000)
    bf.set_option(bsf.BSF_BATCH_OPT_TEST_WITHHOLD, 1)
    bf.run(bsf.BSF_BATCH_PERSISTENT)
    assert bf.status() == bsf.BSF_ETIMEOUT
    bf.set_option(bsf.BSF_BATCH_OPT_TEST_WITHHOLD, 0)
    bf.set_option(bsf.BSF_BATCH_OPT_WAIT_LIMIT, 1 << 22)
    bf.run(bsf.BSF_BATCH_PERSISTENT | bsf.BSF_BATCH_GRAPH)
    assert bf.status() == 0
    for o, r in zip(d_outs, _refs(imgs, covs, 2, info.frac_bits)):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    bf.close()


def test_autotuned_persistent_launch_and_tune_cache(tmp_path):
    # the tuner's choices lie in its candidate sets, are written to the tune
    # cache and read back by a new batch (which then tunes nothing)
    from paper_1109_5114_gb300 import bsf
    imgs, covs, vmax, _, d_imgs, d_covs, d_outs = _small_batch(2, seed0=4, count=6)
    cache = str(tmp_path / "tune.txt")
    bf = bsf.BatchFilter(2, "symmetric", frac_bits=-1, value_bound=vmax)
    bf.set_tune_cache(cache)
    info = bf.plan(d_imgs, d_covs, d_outs, autotune=True)
    assert info.rows_per_item in (1, 2, 4, 8) and info.stencil_tile_rows in (8, 16, 32)
    assert all(c in (32, 48, 64, 96, 128) for c in info.scan_chunk)
    bf.run(bsf.BSF_BATCH_PERSISTENT | bsf.BSF_BATCH_GRAPH)
    assert bf.status() == 0
    for o, r in zip(d_outs, _refs(imgs, covs, 2, info.frac_bits)):
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    bf.close()
    bf2 = bsf.BatchFilter(2, "symmetric", frac_bits=-1, value_bound=vmax)
    bf2.set_tune_cache(cache)
    info2 = bf2.plan(d_imgs, d_covs, d_outs, autotune=True)
    assert (info2.rows_per_item, info2.stencil_tile_rows, info2.persist_grid) == \
        (info.rows_per_item, info.stencil_tile_rows, info.persist_grid)
    assert list(info2.scan_chunk) == list(info.scan_chunk)
    bf2.close()
