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
        own, recvs = bands.halo_exchange(torch.from_numpy(acc_band[a0:a1].copy()), H, R, rank, world)
        own = own.numpy().view(np.uint64)
        for start, buf in recvs:           # the oracle's add (the library's on a GPU)
            own[start:start + buf.shape[0]] += buf.numpy().view(np.uint64)
        whole = ob.adjoint_modular_acc(g, L, n, boundary, R)
        np.testing.assert_array_equal(own.view(np.int64), whole[y0:y1])
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


def _pairs(acc_obj):
    """Python-integer sums as int128 two's complement (low, high) int64 pairs."""
    H, W = acc_obj.shape
    out = np.zeros((H, W, 2), dtype=np.uint64)
    for y in range(H):
        for x in range(W):
            v = int(acc_obj[y, x]) & ((1 << 128) - 1)
            out[y, x, 0] = v & ((1 << 64) - 1)
            out[y, x, 1] = v >> 64
    return out.view(np.int64)


def _add128(a, b):
    """(low, high) int64 pairs added modulo 2^128 (the oracle's form of the
    library's 128-bit halo add)."""
    au, bu = a.view(np.uint64), b.view(np.uint64)
    lo = au[..., 0] + bu[..., 0]
    carry = (lo < au[..., 0]).astype(np.uint64)
    hi = au[..., 1] + bu[..., 1] + carry
    return np.stack([lo, hi], axis=-1).view(np.int64)


def _worker_d2(rank, world, port, H, W, boundary):
    import torch.distributed as dist
    import workloads as wl
    from oracle import config
    from oracle import continuous as cn
    from paper_1109_5114_gb300 import bands
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 2
        gout = wl.uniform_image(H, W, seed=14, lo=-1.0, hi=1.0).astype(np.float32)
        planes = wl.param_fields_logsig_theta_logrho(H, W, 15, logsig_range=(-1.0, 0.5), logrho_range=(0.0, 1.0))
        R = config.padding(planes, n, "d2", kind=1)
        bands.check_bands(H, R, world)
        y0, y1 = bands.band_bounds(H, world, rank)
        qg = cn.grad_frac_bits_d2(float(np.abs(gout).max()))
        pix = [(y, x) for y in range(H) for x in range(W)]
        recs = cn.filter_d2_direct(np.zeros((H, W), dtype=np.int64), planes, n, boundary, pix, kind=1, R=R)
        gq = {p: cn.quantize_weight_d2(float(gout[p]), recs[p]["M"], qg) for p in pix}
        band = cn.adjoint_d2_acc({p: v for p, v in gq.items() if y0 <= p[0] < y1}, planes, n, boundary,
                                 (H, W), kind=1, R=R)
        a0, a1 = bands.halo_rows(H, R, y0, y1)
        own, recvs = bands.halo_exchange(torch.from_numpy(_pairs(band[a0:a1])), H, R, rank, world)
        own = own.numpy()
        for start, buf in recvs:
            own[start:start + buf.shape[0]] = _add128(own[start:start + buf.shape[0]], buf.numpy())
        whole = cn.adjoint_d2_acc(gq, planes, n, boundary, (H, W), kind=1, R=R)
        np.testing.assert_array_equal(own, _pairs(whole[y0:y1]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,boundary", [(2, 2), (3, 0)])
def test_band_backward_halo_exchange_continuous_steps(world, boundary):
    # the 128-bit adjoint sums of the continuous steps travel as int64 pairs
    H, W = 54, 12
    torch.multiprocessing.spawn(_worker_d2, args=(world, _free_port(), H, W, boundary), nprocs=world, join=True)
