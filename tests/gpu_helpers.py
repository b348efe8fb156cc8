"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs.

The configuration of a run (the padding R, the automatic fraction bits q and
element width) is computed by the oracle (oracle.config) and checked against
the library's choice before any output is compared; nothing the CUDA path
chose is fed into the oracle."""
import numpy as np

from oracle import config, kernels, modular, params
from oracle.rounding import quantize


# step rules, direction sets and element widths of the C ABI's codes
RULES = {0: "corrected", 1: "paper", 2: "d2", 3: "sampled"}
DIRS = {0: "cartesian", 1: "second", 2: "pair"}
WIDTHS = {0: None, 1: 64, 2: 128, 5: 32}


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
    # R and q by the oracle's rules, checked against the library's choice
    rule = RULES[step_rule]
    dirs = DIRS[directions]
    R = oracle_R(cov, n, rule, dirs, gpu=info.R, max_reach=max_reach)
    if precision in (3, 4):       # floating-point running sums hold the values themselves
        q_or = 0
        assert info.frac_bits == 0
    else:
        bits, q_or = oracle_q(img, cov, n, q, WIDTHS[precision], rule, dirs, gpu=info.frac_bits)
        assert info.elem_bytes * 8 == bits, (info.elem_bytes, bits)
    res = dict(out=out.cpu().numpy(), R=R, q=q_or, info=info, status=st)
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


def oracle_R(cov, n, rule="corrected", dirs="cartesian", kind=0, gpu=None, max_reach=-1):
    """The padding R by the oracle's rule (or the test's own explicit bound);
    with gpu given, asserts that the library chose the same."""
    R = max_reach if max_reach >= 0 else config.padding(cov, n, rule, dirs, kind)
    if gpu is not None:
        got = gpu["R"] if isinstance(gpu, dict) else gpu
        assert got == R, f"library padding R = {got}, oracle rule {R}"
    return R


def oracle_R_two_pass(cov, n, frac=0.5, kind=0, gpu=None):
    """Algorithm 1's padding: the oracle's R over both fields of the split
    (the isotropic sigma^2 I and the residual C - sigma^2 I)."""
    from oracle import continuous, two_pass
    C = np.stack(continuous.covariance_planes(cov, kind)).astype(np.float32)
    iso, res = two_pass.split_field(C, two_pass.sigma2_global(C, frac))
    R = max(config.padding(iso, n), config.padding(res, n))
    if gpu is not None:
        assert gpu == R, f"library padding R = {gpu}, oracle rule {R}"
    return R


def oracle_q(img, cov, n, frac_bits, bits=64, rule="corrected", dirs="cartesian", kind=0, gpu=None,
             vmax=None):
    """(bits, q) by the oracle's rule (bits None: automatic width); with gpu
    given, asserts that the library chose the same q."""
    mass = config.mass_bound(cov, n, rule, dirs, kind)
    b, q = config.resolve(img, mass, frac_bits, bits, continuous=(rule == "d2"), vmax=vmax,
                          wide_only=rule in ("d2", "sampled"))
    if gpu is not None:
        got = gpu["q"] if isinstance(gpu, dict) else gpu
        assert got == q, f"library q = {got}, oracle rule {q}"
    return b, q


def run_oracle(img, cov, n, boundary, q, R=None, bits=64, out_dtype=np.float32, rule="corrected", gpu=None,
               max_reach=-1):
    """The modular oracle with the oracle's own R (or the test's explicit
    max_reach); with gpu given, the library's R must equal it."""
    if R is None:
        R = oracle_R(cov, n, rule, gpu=gpu, max_reach=max_reach)
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
