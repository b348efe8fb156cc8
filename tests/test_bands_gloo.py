"""The multi-device row-band backward on CPU ranks (gloo, world sizes 2 and
3): each rank takes the oracle's adjoint of its band alone, keeps the rows
that adjoint reaches, and runs the halo add-exchange and the scale
all-reduce of paper_1109_5114_gb300/bands.py; its own rows must then equal
the whole-image adjoint exactly.  Checks the host side of the N > 1 path (the
band kernels themselves are checked on one GPU in test_gpu_bands.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(H, W, n):
    import workloads as wl
    from oracle import params
    gout = wl.uniform_image(H, W, seed=4, lo=-1.0, hi=1.0).astype(np.float32)
    cov = wl.random_cov_field(H, W, seed=6, sigma_range=(0.5, 2.5), rho_range=(1.0, 3.0))
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], n)
    R = max(int(params.reach(L, n).max()), 3 * n)
    return gout, L, R


def _worker(rank, world, port, H, W, n, boundary):
    import torch.distributed as dist
    from oracle import backward as ob
    from oracle import modular
    from paper_1109_5114_gb300 import bands
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gout, L, R = _inputs(H, W, n)
        bands.check_bands(H, R, world)
        y0, y1 = bands.band_bounds(H, world, rank)
        qg = bands.common_grad_bits(float(np.abs(gout[y0:y1]).max()))
        assert qg == ob.grad_frac_bits(float(np.abs(gout).max()))
        D = modular.masses(L, n)
        g = ob.quantize_weights(gout, D, qg)
        g_band = np.zeros_like(g)
        g_band[y0:y1] = g[y0:y1]
        acc_band = ob.adjoint_modular_acc(g_band, L, n, boundary, R)
        a0, a1 = bands.halo_rows(H, R, y0, y1)
        # the band's adjoint reaches no row outside [a0, a1)
        assert not acc_band[:a0].any() and not acc_band[a1:].any()
        own = bands.halo_exchange_add(torch.from_numpy(acc_band[a0:a1].copy()), H, R, rank, world)
        whole = ob.adjoint_modular_acc(g, L, n, boundary, R)
        np.testing.assert_array_equal(own.numpy(), whole[y0:y1])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,boundary", [(2, 2, 2), (3, 1, 0), (2, 3, 1), (3, 2, 2)])
def test_band_backward_halo_exchange(world, n, boundary):
    H, W = 64, 24
    _, _, R = _inputs(H, W, n)
    assert H // world >= R
    torch.multiprocessing.spawn(_worker, args=(world, _free_port(), H, W, n, boundary),
                                nprocs=world, join=True)


def test_band_bounds_cover_rows_once():
    from paper_1109_5114_gb300 import bands
    for H in (1, 7, 64, 2048, 2049):
        for world in (1, 2, 3, 8):
            if world > H:
                continue
            spans = [bands.band_bounds(H, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == H
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    with pytest.raises(ValueError):
        bands.check_bands(100, 40, 3)
