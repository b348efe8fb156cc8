"""Precision study of the running-sum arithmetic (the 8192^2 uint8, n = 3
workload): the same filter with uint128 and uint64 fixed-point running sums,
float64 running sums and compensated float32 (double-float) running sums,
float32 output; max and RMS relative error of each against the exact
definition at sampled pixels.  The fixed-point paths must be exact (uint64
only where its bound holds, which the library checks); the floating-point
ones are recorded as measured (run with -s to print the table)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import kernels, params
from oracle.rounding import quantize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _run(img, cov, n, precision, q):
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = img.shape
    f = bsf.BoxSplineFilter(H, W, n, "symmetric", precision=precision, frac_bits=q)
    tc = torch.from_numpy(cov).cuda()
    f.plan(tc)
    out = f.filter(torch.from_numpy(img).cuda(), tc)
    torch.cuda.synchronize()
    st = f.status()
    res = out.cpu().numpy()
    f.close()
    return res, st


def _errors(out, ref):
    rel = [abs(float(out[p]) - v) / abs(v) if v != 0 else abs(float(out[p])) for p, v in ref.items()]
    rel = np.array(rel)
    if not np.isfinite(rel).all():
        return math.inf, math.inf, int((~np.isfinite(rel)).sum())
    return float(rel.max()), float(np.sqrt((rel ** 2).mean())), 0


def test_precision_study_8192_u8_n3():
    from paper_1109_5114_gb300 import bsf
    H = W = 8192
    n = 3
    img = wl.blob_image_u8(H, W, seed=0)
    cov = wl.random_cov_field(H, W, seed=0, sigma_range=(2.0, 32.0), rho_range=(1.0, 3.0))
    rng = np.random.default_rng(5)
    pix = sorted({(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(40)})
    ys = np.array([p[0] for p in pix]); xs = np.array([p[1] for p in pix])
    sub = cov[:, ys, xs][:, :, None]
    L = params.integer_steps(sub[0], sub[1], sub[2], n)[0][:, :, 0]
    Lfield = np.zeros((4, H, W), dtype=np.int64)
    Lfield[:, ys, xs] = L
    keep = [p for i, p in enumerate(pix) if kernels.kernel_mass(L[:, i], n) < (1 << 62)]
    acc = kernels.correlate_exact_sampled(quantize(img, 0), Lfield, n, 2, keep)
    ref = {p: acc[p] / kernels.kernel_mass(Lfield[:, p[0], p[1]], n) for p in keep}
    rows = []
    for name, prec in [("uint128", bsf.BSF_FIX128), ("uint64", bsf.BSF_FIX64),
                       ("float64", bsf.BSF_F64ACC), ("float32-compensated", bsf.BSF_F32KAHAN)]:
        out, st = _run(img, cov, n, prec, 0)
        mx, rms, bad = _errors(out, ref)
        rows.append((name, st, mx, rms, bad))
        if prec == bsf.BSF_FIX128:
            assert st == 0 and mx <= 2.0 ** -23
        if prec == bsf.BSF_FIX64:
            # exact where prod L^3 * 255 < 2^63, flagged otherwise
            assert st in (0, bsf.BSF_EOVERFLOW)
            if st == 0:
                assert mx <= 2.0 ** -23
    print("\nprecision study, 8192^2 u8, n=3, %d sampled pixels" % len(keep))
    print("%-22s %8s %14s %14s %10s" % ("running sums", "status", "max rel err", "rms rel err", "non-finite"))
    for r in rows:
        print("%-22s %8d %14.3e %14.3e %10d" % r)


def test_float64_sums_are_accurate_at_small_sizes():
    # 256^2 float64 image, n = 1, C = 16 I: float64 running sums stay within
    # ~1e-9 relative (the n-fold growth is still small)
    from paper_1109_5114_gb300 import bsf
    H = W = 256
    img = wl.uniform_image(H, W, seed=0)
    cov = wl.constant_cov_field(H, W, 16.0, 0.0, 16.0)
    L, _ = params.integer_steps(cov[0], cov[1], cov[2], 1)
    pix = [(0, 0), (17, 200), (128, 128), (255, 3), (90, 91)]
    exact = kernels.correlate_f64(img, L, 1, 2, pixels=pix)
    for prec, tol in [(bsf.BSF_F64ACC, 1e-9), (bsf.BSF_F32KAHAN, 1e-5)]:
        out, st = _run(img, cov, 1, prec, 0)
        assert st == 0
        for p in pix:
            assert abs(float(out[p]) - exact[p]) <= tol * abs(exact[p]) + 2e-7 * abs(exact[p])
