"""Row-band decomposition of one image over several devices, one process per
device (torch.distributed: NCCL between GPUs, gloo on CPU).

Forward: rank r filters image rows [y0, y1) of its band from running sums
that restart R rows above it (``BoxSplineFilter.filter_rows``); every tap of
a band pixel lies in the band's padded rows, so the band equals the
whole-image result bit for bit and no data is exchanged.

Backward (image gradient): the adjoint of a band reaches R rows beyond it on
each side.  Each rank computes its band's adjoint as exact int64 sums on rows
[a0, a1) = [y0 - R, y1 + R) clipped to the image (``backward_rows``); one
all-reduce of max |gout| fixes the common fixed-point scale of the gradient
weights, and a halo add-exchange of those R rows with each neighbour
completes the rows [y0, y1) the rank owns, which the library then rounds
(``grad_finalize``).  The integer sums make the assembled gradient equal the
single-device backward bit for bit.

The host logic here is argument marshalling and message passing only; every
arithmetic step of the filter runs in the library's kernels.
"""
from __future__ import annotations


def band_bounds(H: int, world: int, rank: int):
    """Rows [y0, y1) of rank's band: H split into world bands differing by at most one row."""
    base, extra = divmod(H, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def halo_rows(H: int, R: int, y0: int, y1: int):
    """Image rows [a0, a1) that a band's adjoint reaches."""
    return max(0, y0 - R), min(H, y1 + R)


def check_bands(H: int, R: int, world: int) -> None:
    """Each halo must reach only the adjacent band: every band at least R rows."""
    shortest = min(b - a for a, b in (band_bounds(H, world, r) for r in range(world)))
    if shortest < R:
        raise ValueError(f"bands of {shortest} rows are shorter than the reach R = {R}; "
                         "use fewer bands")


def halo_exchange(acc, H: int, R: int, rank: int, world: int, group=None):
    """Send this band's halo rows to the neighbours and receive theirs.

    acc: int64 tensor [a1 - a0][W] of the band's adjoint sums, or [a1 - a0][W][2]
    for 128-bit sums as (low, high) pairs (CPU or CUDA, as the process group's
    backend requires).  Rows [a0, y0) go to rank - 1 and
    rows [y1, a1) to rank + 1; the matching rows of the neighbours are
    received.  Returns (own, recvs): own is a copy of the own rows [y0, y1),
    recvs a list of (first own row, received rows) that still have to be
    added to own (two's complement, wrapping like the library's modular
    sums: the library's bsf_grad_halo_add does that on the device)."""
    import torch
    import torch.distributed as dist
    y0, y1 = band_bounds(H, world, rank)
    a0, a1 = halo_rows(H, R, y0, y1)
    own = acc[y0 - a0:y1 - a0].clone()
    ops, recvs = [], []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, acc[:y0 - a0].contiguous(), rank - 1, group))
        n_up = min(H, y0 + R) - y0                 # rank - 1's rows below its band
        buf = torch.empty((n_up,) + tuple(acc.shape[1:]), dtype=acc.dtype, device=acc.device)
        ops.append(dist.P2POp(dist.irecv, buf, rank - 1, group))
        recvs.append((0, buf))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, acc[y1 - a0:].contiguous(), rank + 1, group))
        n_dn = y1 - max(0, y1 - R)                 # rank + 1's rows above its band
        buf = torch.empty((n_dn,) + tuple(acc.shape[1:]), dtype=acc.dtype, device=acc.device)
        ops.append(dist.P2POp(dist.irecv, buf, rank + 1, group))
        recvs.append((y1 - y0 - n_dn, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return own, recvs


def common_grad_bits(local_max: float, group=None, device="cpu", filt=None) -> int:
    """All-reduce (max) of the bands' max |gout|, then the library's scale rule
    (the context's: 64- or 128-bit adjoint sums; without a context the 64-bit
    rule)."""
    import torch
    import torch.distributed as dist
    from . import bsf
    t = torch.tensor([local_max], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    m = float(t.item())
    return filt.grad_frac_bits(m) if filt is not None else int(bsf.bsf_grad_frac_bits(m))


def backward_bands(filt, gout, cov, rank: int, world: int, group=None):
    """Image gradient rows [y0, y1) of this rank's band (float32 CUDA tensor).

    gout and cov are the whole-image tensors (only the band's rows of gout
    and the band's halo rows of cov are read)."""
    info = filt.info()
    check_bands(filt.H, info.R, world)
    y0, y1 = band_bounds(filt.H, world, rank)
    qg = common_grad_bits(filt.grad_absmax_rows(gout, y0, y1), group, device=gout.device, filt=filt)
    acc, _, _ = filt.backward_rows(gout, cov, y0, y1, qg)
    own, recvs = halo_exchange(acc, filt.H, info.R, rank, world, group)
    for start, buf in recvs:
        filt.grad_halo_add(own[start:start + buf.shape[0]], buf)
    return filt.grad_finalize(own, qg)
