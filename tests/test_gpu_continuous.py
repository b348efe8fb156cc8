"""GPU parity of the continuous-step filter (interpolated taps) and of its
Jacobian with respect to the covariance field, through the C ABI, against
oracle/continuous.py.

Outputs of the fixed-point path are compared bit for bit with the oracle's
running-sum pipeline (same quantisation, same integer sums, same final
rounding).  The Jacobian is float (exact integer derivative sums, float64
combination, float32 chain rule on the GPU; exact rationals and a float64
complex-step chain in the oracle), compared with the tolerance
|J_gpu - J_oracle| <= 2e-4 max|J_oracle| + 1e-3 |J_oracle| per plane: the
float32 chain carries a few units of 2^-24 per step, amplified at most by the
cancellation in the implicit derivative of the scale solve.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import continuous as cn
from oracle import kernels
from tests.gpu_helpers import oracle_R, oracle_q

pytestmark = pytest.mark.gpu

ATOL_REL, RTOL = 2e-4, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def _fields(H, W, seed, kind, smax=2.5, rmax=3.0):
    if kind == 0:
        return wl.random_cov_field(H, W, seed=seed, sigma_range=(0.3, smax), rho_range=(1.0, rmax))
    return wl.param_fields_logsig_theta_logrho(H, W, seed, logsig_range=(-1.0, math.log(smax)),
                                               logrho_range=(0.0, math.log(rmax)))


def _filter(H, W, n, boundary, q, precision, kind, max_reach=-1):
    from paper_1109_5114_gb300 import bsf
    return bsf.BoxSplineFilter(H, W, n, boundary, max_reach=max_reach, precision=precision,
                               frac_bits=q, step_rule=2, cov_kind=kind)


def _run(img, planes, n, boundary, q, precision, kind, out_dtype=np.float32, jac=False,
         max_reach=-1):
    import torch
    H, W = img.shape
    f = _filter(H, W, n, boundary, q, precision, kind, max_reach)
    ti = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    tc = torch.from_numpy(np.ascontiguousarray(planes, dtype=np.float32)).cuda()
    if jac:
        out, J = f.filter_jacobian(ti, tc)
    else:
        out = f.filter(ti, tc, out_dtype=torch.float32 if out_dtype == np.float32 else torch.float64)
        J = None
    torch.cuda.synchronize()
    st = f.status()
    info = f.info()
    # R and q by the oracle's rules, checked against the library's choice
    R = oracle_R(planes, n, "d2", kind=kind, gpu=info.R, max_reach=max_reach)
    bits, q_or = oracle_q(img, planes, n, q, 64 if precision == 1 else 128, "d2", kind=kind, gpu=info.frac_bits)
    return dict(out=out.cpu().numpy(), jac=None if J is None else J.cpu().numpy(), R=R,
                q=q_or, status=st, filt=f, img=ti, cov=tc)


def _sample(H, W, k, seed):
    rng = np.random.default_rng(seed)
    pts = {(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (H // 2, W // 2)}
    pts |= {(0, int(x)) for x in rng.integers(0, W, 6)} | {(H - 1, int(x)) for x in rng.integers(0, W, 6)}
    pts |= {(int(y), 0) for y in rng.integers(0, H, 6)} | {(int(y), W - 1) for y in rng.integers(0, H, 6)}
    while len(pts) < k:
        pts.add((int(rng.integers(0, H)), int(rng.integers(0, W))))
    return sorted(pts)


CASES = [(1, 0, 1, 0), (1, 1, 2, 1), (1, 2, 2, 0), (2, 0, 2, 1), (2, 1, 1, 0), (2, 2, 2, 0),
         (2, 2, 2, 1), (2, 1, 2, 1)]


@pytest.mark.parametrize("n,boundary,prec,kind", CASES)
def test_forward_bit_exact(n, boundary, prec, kind):
    H, W = 21, 70   # several warps per row, ragged last block
    if prec == 1:   # uint64: small kernels and integer values so that q = 0 fits
        img = wl.random_integer_image(H, W, seed=n + boundary, lo=-30, hi=30).astype(np.float64)
        planes = _fields(H, W, seed=3 + n, kind=kind, smax=1.2)
        q = 0
    else:
        img = wl.blob_image(H, W, seed=n, n_blobs=8, sigma_range=(2.0, 8.0))
        planes = _fields(H, W, seed=5 + n, kind=kind)
        q = -1
    for out_dtype in (np.float32, np.float64):
        g = _run(img, planes, n, boundary, q, prec, kind, out_dtype=out_dtype)
        assert g["status"] == 0
        pix = _sample(H, W, 300, seed=n)
        bits = 64 if prec == 1 else 128
        rec = cn.filter_d2_modular(img, planes, n, boundary, g["q"], bits=bits, kind=kind, R=g["R"],
                                   pixels=pix)
        ref = np.array([cn.output(rec[p], g["q"], out_dtype) for p in pix], dtype=out_dtype)
        got = np.array([g["out"][p] for p in pix], dtype=out_dtype)
        np.testing.assert_array_equal(got, ref)


def _check_jac(got, ref):
    for c in range(3):
        scale = np.abs(ref[:, c]).max()
        err = np.abs(got[:, c] - ref[:, c])
        assert (err <= ATOL_REL * scale + RTOL * np.abs(ref[:, c])).all(), (c, err.max(), scale)


@pytest.mark.parametrize("n,kind,boundary", [(2, 0, 2), (2, 1, 1), (1, 1, 2), (1, 0, 0)])
def test_jacobian_matches_oracle(n, kind, boundary):
    H, W = 24, 40
    img = wl.blob_image(H, W, seed=7, n_blobs=10, sigma_range=(1.5, 6.0))
    planes = _fields(H, W, seed=11, kind=kind)
    g = _run(img, planes, n, boundary, -1, 2, kind, jac=True)
    assert g["status"] == 0
    pix = _sample(H, W, 160, seed=2)
    rec = cn.filter_d2_modular(img, planes, n, boundary, g["q"], bits=128, kind=kind, R=g["R"],
                               pixels=pix)
    # forward of the Jacobian call is the forward
    ref_out = np.array([cn.output(rec[p], g["q"]) for p in pix], dtype=np.float32)
    np.testing.assert_array_equal(np.array([g["out"][p] for p in pix]), ref_out)
    ref = np.array([cn.jacobian_planes(rec[p], planes[:, p[0], p[1]].astype(np.float64), kind, n, g["q"])
                    for p in pix])
    got = np.array([g["jac"][:, p[0], p[1]] for p in pix])
    _check_jac(got, ref)


def test_jacobian_at_clamped_scales():
    # anisotropy up to 8 (beyond the elongation bound in places): the scale
    # solve sits on its bounds (a zero scale, or C12 clamped to e(phi))
    H, W = 24, 40
    img = wl.blob_image(H, W, seed=8, n_blobs=10, sigma_range=(1.5, 6.0))
    planes = wl.random_cov_field(H, W, seed=3, sigma_range=(0.5, 3.0), rho_range=(1.0, 8.0))
    g = _run(img, planes, 2, kernels.SYMMETRIC, -1, 2, 0, jac=True)
    assert g["status"] == 0 and g["filt"].info().clamp_count > 0
    pix = _sample(H, W, 160, seed=4)
    rec = cn.filter_d2_modular(img, planes, 2, kernels.SYMMETRIC, g["q"], bits=128, R=g["R"],
                               pixels=pix)
    ref = np.array([cn.jacobian_planes(rec[p], planes[:, p[0], p[1]].astype(np.float64), 0, 2, g["q"])
                    for p in pix])
    _check_jac(np.array([g["jac"][:, p[0], p[1]] for p in pix]), ref)


def test_constant_image_has_zero_jacobian():
    H, W = 20, 33
    img = np.full((H, W), 37.0, dtype=np.float32)
    planes = _fields(H, W, seed=4, kind=1)
    g = _run(img, planes, 2, kernels.SYMMETRIC, -1, 2, 1, jac=True)
    assert g["status"] == 0
    # float32 rule RN32(RN32(acc) 2^-q) / RN32(M): within 1.5 ulp of 37
    assert np.abs(g["out"] - 37.0).max() <= 1.5 * np.spacing(np.float32(37.0))
    assert np.abs(g["jac"]).max() < 1e-9


def test_backward_recompute_equals_stored_jacobian_product():
    import torch
    H, W = 30, 45
    img = wl.blob_image(H, W, seed=2, n_blobs=9, sigma_range=(2.0, 6.0))
    planes = _fields(H, W, seed=12, kind=1)
    g = _run(img, planes, 2, kernels.SYMMETRIC, -1, 2, 1, jac=True)
    f = g["filt"]
    gout = torch.from_numpy(wl.uniform_image(H, W, seed=3, lo=-1, hi=1).astype(np.float32)).cuda()
    via_jac = f.jacobian_vjp(gout, torch.from_numpy(g["jac"]).cuda())
    _, via_recompute = f.backward(gout, g["cov"], want_gcov=True, want_gimg=False)
    torch.cuda.synchronize()
    assert f.status() == 0
    np.testing.assert_array_equal(via_recompute.cpu().numpy(), via_jac.cpu().numpy())
    np.testing.assert_array_equal(via_jac.cpu().numpy(), gout.cpu().numpy()[None] * g["jac"])


def test_autograd_parameter_gradient():
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = 26, 38
    img = torch.from_numpy(wl.blob_image(H, W, seed=1, n_blobs=9, sigma_range=(2.0, 6.0))).cuda()
    planes = _fields(H, W, seed=13, kind=1)
    target = torch.from_numpy(wl.uniform_image(H, W, seed=5, lo=0, hi=1).astype(np.float32)).cuda()
    f = _filter(H, W, 2, kernels.SYMMETRIC, -1, 2, 1)
    p = torch.from_numpy(planes).cuda().requires_grad_(True)
    out = bsf.box_spline_filter(img, p, f)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    out2, J = f.filter_jacobian(img, p.detach())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.detach().cpu().numpy(), out2.cpu().numpy())
    expect = ((out2 - target)[None] * J).cpu().numpy()
    np.testing.assert_array_equal(p.grad.cpu().numpy(), expect)
    # no covariance gradient requested: plain forward, no Jacobian
    out3 = bsf.box_spline_filter(img, p.detach(), f)
    np.testing.assert_array_equal(out3.cpu().numpy(), out2.cpu().numpy())


def test_out_of_reach_pixels_take_identity_steps():
    from paper_1109_5114_gb300 import bsf
    H, W = 18, 40
    img = wl.random_integer_image(H, W, seed=9, lo=-100, hi=100).astype(np.float32)
    planes = wl.constant_cov_field(H, W, 0.3, 0.0, 0.3)   # reach 9: inside
    planes[:, 5:9, 10:20] = np.array([30.0, 0.0, 30.0], dtype=np.float32)[:, None, None]
    g = _run(img, planes, 2, kernels.SYMMETRIC, 8, 2, 0, jac=True, max_reach=9)
    assert g["R"] == 9 and g["status"] == bsf.BSF_ERANGE
    pix = [(6, 12), (7, 19), (0, 0), (12, 30)]
    rec = cn.filter_d2_modular(img, planes, 2, kernels.SYMMETRIC, 8, bits=128, R=9, pixels=pix)
    assert rec[(6, 12)]["far"] and not rec[(0, 0)]["far"]
    for p in pix:
        assert g["out"][p] == cn.output(rec[p], 8)
    assert g["out"][6, 12] == img[6, 12]
    assert (g["jac"][:, 6, 12] == 0).all()


def test_argument_errors():
    import torch
    from paper_1109_5114_gb300 import bsf
    with pytest.raises(bsf.BsfError):
        bsf.BoxSplineFilter(16, 16, 3, step_rule=2)
    H, W = 16, 20
    img = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    cov = torch.from_numpy(wl.constant_cov_field(H, W, 2.0, 0.0, 2.0)).cuda()
    f = bsf.BoxSplineFilter(H, W, 2, precision=bsf.BSF_F64ACC, step_rule=2)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f = bsf.BoxSplineFilter(H, W, 2, max_reach=6, precision=2, step_rule=2)
    with pytest.raises(bsf.BsfError):
        f.filter(img, cov)
    f = bsf.BoxSplineFilter(H, W, 2, precision=2, step_rule=0)
    with pytest.raises(bsf.BsfError):
        f.filter_jacobian(img, cov)
    # a uint64 context takes the 128-bit image gradient too; asking for no
    # gradient at all is an error
    f = bsf.BoxSplineFilter(H, W, 2, precision=1, frac_bits=4, step_rule=2)
    f.filter(img, cov)
    gout = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    gimg, gcov = f.backward(gout, cov, want_gimg=True, want_gcov=True)
    torch.cuda.synchronize()
    assert f.status() == 0 and (gimg == 0).all() and (gcov == 0).all()
    with pytest.raises(bsf.BsfError):
        f.backward(gout, cov, want_gimg=False, want_gcov=False)


def test_log_parameter_field_in_the_integer_step_filter():
    # the same pixels through cov_kind 1 and through the float32 covariance the
    # oracle builds from the log parameters: identical steps, identical output
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = 40, 52
    img = torch.from_numpy(wl.blob_image(H, W, seed=3, n_blobs=8)).cuda()
    planes = wl.param_fields_logsig_theta_logrho(H, W, 21, logsig_range=(0.0, 2.0))
    C = np.stack(cn.cov_from_log_params(planes[0], planes[1], planes[2]))
    outs = []
    for kind, field in ((1, planes), (0, C)):
        f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=1, frac_bits=20, cov_kind=kind)
        outs.append(f.filter(img, torch.from_numpy(np.ascontiguousarray(field)).cuda()).cpu().numpy())
        assert f.status() == 0
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n,boundary,kind", [(2, 2, 1), (2, 0, 0), (1, 1, 1), (2, 1, 0)])
def test_image_gradient_bit_exact(n, boundary, kind):
    import torch
    from oracle.rounding import rn_f32_int
    H, W = 22, 45
    planes = _fields(H, W, seed=15 + n, kind=kind)
    gout = wl.uniform_image(H, W, seed=16, lo=-1, hi=1).astype(np.float32)
    f = _filter(H, W, n, boundary, -1, 2, kind)
    tc = torch.from_numpy(planes).cuda()
    f.plan(tc)
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tc, want_gimg=True, want_gcov=False)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = oracle_R(planes, n, "d2", kind=kind, gpu=f.info().R)
    qg = cn.grad_frac_bits_d2(float(np.abs(gout).max()))
    pix = [(y, x) for y in range(H) for x in range(W)]
    recs = cn.filter_d2_direct(np.zeros((H, W), dtype=np.int64), planes, n, boundary, pix, kind=kind, R=R)
    gq = {p: cn.quantize_weight_d2(float(gout[p]), recs[p]["M"], qg) for p in pix}
    acc = cn.adjoint_d2_acc(gq, planes, n, boundary, (H, W), kind=kind, R=R)
    ref = np.array([[np.float32(rn_f32_int(acc[y, x]) * np.float32(2.0 ** -qg)) for x in range(W)]
                    for y in range(H)], dtype=np.float32)
    np.testing.assert_array_equal(gimg.cpu().numpy(), ref)


def _window_case_field(case, H, W):
    if case == "one_pass":     # sigma 0.5-2: every block's samples fit one window
        return wl.random_cov_field(H, W, seed=31, sigma_range=(0.5, 2.0), rho_range=(1.0, 2.0))
    if case == "row_bands":    # sigma 12-15: windows of several row bands
        return wl.random_cov_field(H, W, seed=33, sigma_range=(12.0, 15.0), rho_range=(1.0, 2.0))
    s2 = np.float32(27.0 ** 2)  # one anisotropic sigma ~ 27: more bands than allowed, direct adds
    return np.stack([np.full((H, W), s2 * np.float32(1.3)), np.full((H, W), s2 * np.float32(0.2)),
                     np.full((H, W), s2)]).astype(np.float32)


@pytest.mark.parametrize("case,H,W", [("one_pass", 24, 70), ("row_bands", 8, 36), ("direct", 8, 36)])
def test_image_gradient_sample_windows(case, H, W):
    # the scatter sums a block's samples in a shared window before adding it
    # to the global sums: small scales fit one window pass, larger ones take
    # several row bands, the largest fall back to direct global adds; every
    # regime gives the oracle's adjoint bit for bit (ragged image sizes)
    import torch
    from oracle.rounding import rn_f32_int
    n, boundary = 2, kernels.SYMMETRIC
    planes = _window_case_field(case, H, W)
    gout = wl.uniform_image(H, W, seed=32, lo=-1, hi=1).astype(np.float32)
    f = _filter(H, W, n, boundary, -1, 2, 0)
    tc = torch.from_numpy(planes).cuda()
    f.plan(tc)
    gimg, _ = f.backward(torch.from_numpy(gout).cuda(), tc, want_gimg=True, want_gcov=False)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = oracle_R(planes, n, "d2", kind=0, gpu=f.info().R)
    qg = cn.grad_frac_bits_d2(float(np.abs(gout).max()))
    pix = [(y, x) for y in range(H) for x in range(W)]
    recs = cn.filter_d2_direct(np.zeros((H, W), dtype=np.int64), planes, n, boundary, pix, kind=0, R=R)
    gq = {p: cn.quantize_weight_d2(float(gout[p]), recs[p]["M"], qg) for p in pix}
    acc = cn.adjoint_d2_acc(gq, planes, n, boundary, (H, W), kind=0, R=R)
    ref = np.array([[np.float32(rn_f32_int(acc[y, x]) * np.float32(2.0 ** -qg)) for x in range(W)]
                    for y in range(H)], dtype=np.float32)
    np.testing.assert_array_equal(gimg.cpu().numpy(), ref)


def test_autograd_image_and_parameter_gradients():
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = 30, 41
    img = torch.from_numpy(wl.blob_image(H, W, seed=4, n_blobs=9, sigma_range=(2.0, 6.0))).cuda()
    planes = torch.from_numpy(_fields(H, W, seed=17, kind=1)).cuda()
    target = torch.from_numpy(wl.uniform_image(H, W, seed=6, lo=0, hi=1).astype(np.float32)).cuda()
    f = _filter(H, W, 2, kernels.SYMMETRIC, -1, 2, 1)
    f.plan(planes)
    x = img.clone().requires_grad_(True)
    p = planes.clone().requires_grad_(True)
    out = bsf.box_spline_filter(x, p, f)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    gout = (out.detach() - target).contiguous()
    gimg, _ = f.backward(gout, planes, want_gimg=True, want_gcov=False)
    _, J = f.filter_jacobian(img, planes)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.grad.cpu().numpy(), gimg.cpu().numpy())
    np.testing.assert_array_equal(p.grad.cpu().numpy(), (gout[None] * J).cpu().numpy())
    # the image gradient is the adjoint: <gout, A d> = <A^T gout, d> for a probe d
    d = torch.from_numpy(wl.uniform_image(H, W, seed=8, lo=-1, hi=1).astype(np.float32)).cuda()
    Ad = f.filter(d, planes)
    lhs = float((gout.double() * Ad.double()).sum())
    rhs = float((gimg.double() * d.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1e-3)


def test_memory_budget_recompute_route_equals_stored_route():
    # above its memory budget the differentiable forward keeps only its
    # inputs; the backward recomputes the running sums and the Jacobian
    # product.  Both routes give the same gradients bit for bit, even when
    # another image went through the filter between forward and backward.
    import torch
    from paper_1109_5114_gb300 import bsf
    H, W = 34, 47
    img = torch.from_numpy(wl.blob_image(H, W, seed=6, n_blobs=9, sigma_range=(2.0, 6.0))).cuda()
    other = torch.from_numpy(wl.blob_image(H, W, seed=7, n_blobs=5, sigma_range=(2.0, 6.0))).cuda()
    planes = torch.from_numpy(_fields(H, W, seed=19, kind=1)).cuda()
    target = torch.from_numpy(wl.uniform_image(H, W, seed=9, lo=0, hi=1).astype(np.float32)).cuda()
    grads = []
    for budget in (None, 0):
        f = bsf.BoxSplineFilter(H, W, 2, "symmetric", precision=bsf.BSF_FIX128, frac_bits=-1, step_rule=2,
                                cov_kind=1, memory_budget=budget)
        assert f.stores_jacobian() == (budget is None)
        f.plan(planes)
        x = img.clone().requires_grad_(True)
        p = planes.clone().requires_grad_(True)
        out = bsf.box_spline_filter(x, p, f)
        assert len(out.grad_fn.saved_tensors) == (3 if budget is None else 2)
        f.filter(other, planes)                 # replaces the held running sums
        loss = 0.5 * ((out - target) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        assert f.status() == 0
        grads.append((out.detach().cpu().numpy(), x.grad.cpu().numpy(), p.grad.cpu().numpy()))
        f.close()
    for a, b in zip(grads[0], grads[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n", [1, 2])
def test_image_gradient_on_64bit_context_equals_128bit(n):
    # the image gradient reads no running sums: a context whose forward keeps
    # uint64 sums takes the same 128-bit adjoint and gives the same gradient
    import torch
    H, W = 26, 39
    planes = _fields(H, W, seed=30 + n, kind=1)
    gout = torch.from_numpy(wl.uniform_image(H, W, seed=31, lo=-1, hi=1).astype(np.float32)).cuda()
    tc = torch.from_numpy(planes).cuda()
    outs = []
    for prec in (1, 2):
        f = _filter(H, W, n, kernels.SYMMETRIC, -1, prec, 1)
        f.plan(tc)
        assert f.info().grad_elem_bytes == 16
        gimg, _ = f.backward(gout, tc, want_gimg=True, want_gcov=False)
        torch.cuda.synchronize()
        assert f.status() == 0
        outs.append(gimg.cpu().numpy())
        f.close()
    np.testing.assert_array_equal(outs[0], outs[1])
