"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
import numpy as np

from oracle import kernels, modular, params
from oracle.rounding import quantize


def torch_mod():
    import torch
    return torch


def run_gpu(img, cov, n, boundary, q, precision=1, out_dtype=np.float32, max_reach=-1,
            step_rule=0, want_S=False, want_steps=False, directions=0):
    """Forward filter on cuda:0; returns dict(out, R, q, info[, S, L]).  With
    directions = BSF_DIRS_PAIR, S is the pair (first set's, second set's)."""
    torch = torch_mod()
    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, boundary, max_reach=max_reach, precision=precision,
                            frac_bits=q, step_rule=step_rule, directions=directions)
    if want_S:  # the fused tiles keep no running sums
        f.set_option(bsf.BSF_OPT_TILES, 0)
    ti = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    tc = torch.from_numpy(np.ascontiguousarray(cov, dtype=np.float32)).cuda()
    tdt = torch.float32 if np.dtype(out_dtype) == np.float32 else torch.float64
    out = f.filter(ti, tc, out_dtype=tdt)
    torch.cuda.synchronize()
    st = f.status()
    info = f.info()
    res = dict(out=out.cpu().numpy(), R=info.R, q=info.frac_bits, info=info, status=st)
    if want_steps:
        L = f.steps().cpu().numpy().astype(np.int64) & 0xFFFF
        res["L"] = L & 0x7FFF if directions == 2 else L
        if directions == 2:
            res["second"] = (L[0] & 0x8000) != 0
    if want_S:
        raw, inf = f.preintegrated()
        raw = raw.cpu().numpy()
        sets = 2 if directions == 2 else 1
        if inf.elem_bytes == 4:
            S = raw.view(np.uint32).reshape(sets, inf.Hp, inf.Wp)
            S = [S[i] for i in range(sets)]
        elif inf.elem_bytes == 8:
            S = raw.view(np.uint64).reshape(sets, inf.Hp, inf.Wp)
            S = [S[i] for i in range(sets)]
        else:
            v = raw.view(np.uint64).reshape(sets, inf.Hp, inf.Wp, 2)
            S = [(v[i, ..., 0].copy(), v[i, ..., 1].copy()) for i in range(sets)]
        res["S"] = S[0] if sets == 1 else tuple(S)
    f.close()
    return res


def run_oracle(img, cov, n, boundary, q, R, bits=64, out_dtype=np.float32, rule="corrected"):
    return modular.filter_modular(img, cov, n, boundary, q=q, bits=bits, out_dtype=out_dtype, R=R,
                                  rule=rule, return_all=True)


def oracle_S(img, n, boundary, q, R, bits):
    fq = quantize(img, q, as_object=(bits == 128))
    fe = kernels.extend_image(fq, R, boundary)
    return modular.preintegrate(fe, n, bits)


def oracle_S_second(img, n, boundary, q, R, bits):
    from oracle import knight
    fq = quantize(img, q, as_object=(bits == 128))
    return knight.preintegrate_k(kernels.extend_image(fq, R, boundary), n, bits)


def oracle_steps(cov, n, rule="corrected"):
    L, fl = params.integer_steps(cov[0], cov[1], cov[2], n, rule)
    return L, fl
