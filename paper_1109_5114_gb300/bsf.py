"""ctypes binding of libbsf.so: the C ABI of include/bsf.h under the same names.

Argument marshalling only: every step of the filter runs in the library's
CUDA kernels.  Importing this module loads the library and fails loudly when
it has not been built (there is no CPU fallback).  The ``BoxSplineFilter``
class wraps a context for torch tensors (device memory and the current
stream come from torch; torch does no arithmetic of the filter).
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
LIB_PATH = os.path.join(_PKG, "lib", "libbsf.so")
HEADER = os.path.join(_ROOT, "include", "bsf.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libbsf.so is not built ({LIB_PATH}); run paper_1109_5114_gb300.build.build() "
        "(nvcc for sm_103a). The filter has no CPU path.")

_lib = ctypes.CDLL(LIB_PATH)


def _constants_from_header(path: str) -> dict:
    consts = {}
    with open(path) as fh:
        for line in fh:
            m = re.match(r"#define\s+(BSF_\w+)\s+\(?(-?\d+)u?\)?", line)
            if m:
                consts[m.group(1)] = int(m.group(2))
    return consts


_C = _constants_from_header(HEADER)
globals().update(_C)

bsf_t = ctypes.c_void_p
c_int, c_ll, c_void_p, c_double = ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_double


class bsf_info_t(ctypes.Structure):
    _fields_ = [("H", c_int), ("W", c_int), ("N", c_int), ("n", c_int), ("boundary", c_int),
                ("R", c_int), ("Hp", c_int), ("Wp", c_int), ("pitch", c_ll),
                ("elem_bytes", c_int), ("precision", c_int), ("frac_bits", c_int),
                ("step_rule", c_int), ("max_reach", c_int), ("max_mass", c_double),
                ("clamp_count", ctypes.c_uint), ("flags", ctypes.c_uint),
                ("workspace_bytes", c_ll), ("grad_elem_bytes", c_int)]


def _fn(name, restype, *argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = list(argtypes)
    return f


bsf_create = _fn("bsf_create", c_int, ctypes.POINTER(bsf_t), c_int, c_int, c_int, c_int, c_int, c_int)
bsf_destroy = _fn("bsf_destroy", None, bsf_t)
bsf_set_stream = _fn("bsf_set_stream", c_int, bsf_t, c_void_p)
bsf_set_precision = _fn("bsf_set_precision", c_int, bsf_t, c_int, c_int)
bsf_set_value_bound = _fn("bsf_set_value_bound", c_int, bsf_t, c_double)
bsf_set_step_rule = _fn("bsf_set_step_rule", c_int, bsf_t, c_int)
bsf_plan = _fn("bsf_plan", c_int, bsf_t, c_void_p, c_int)
bsf_preintegrate = _fn("bsf_preintegrate", c_int, bsf_t, c_void_p, c_int, c_ll)
bsf_filter = _fn("bsf_filter", c_int, bsf_t, c_void_p, c_int, c_ll, c_void_p, c_int, c_void_p, c_int, c_ll)
bsf_status = _fn("bsf_status", c_int, bsf_t)
bsf_last_error = _fn("bsf_last_error", ctypes.c_char_p, bsf_t)
bsf_get_info = _fn("bsf_get_info", c_int, bsf_t, ctypes.POINTER(bsf_info_t))
bsf_copy_steps = _fn("bsf_copy_steps", c_int, bsf_t, c_void_p)
bsf_copy_preintegrated = _fn("bsf_copy_preintegrated", c_int, bsf_t, c_void_p)
bsf_set_profiling = _fn("bsf_set_profiling", c_int, bsf_t, c_int)
bsf_set_option = _fn("bsf_set_option", c_int, bsf_t, c_int, c_ll)
bsf_filter_rows = _fn("bsf_filter_rows", c_int, bsf_t, c_void_p, c_int, c_ll, c_void_p, c_int,
                      c_void_p, c_int, c_ll, c_int, c_int)
bsf_filter_backward = _fn("bsf_filter_backward", c_int, bsf_t, c_void_p, c_ll, c_void_p, c_int,
                          c_void_p, c_ll, c_void_p)
bsf_read_profile = _fn("bsf_read_profile", c_int, bsf_t, ctypes.POINTER(c_double), ctypes.POINTER(c_int))
bsf_filter_jacobian = _fn("bsf_filter_jacobian", c_int, bsf_t, c_void_p, c_int, c_ll, c_void_p, c_int,
                          c_void_p, c_int, c_ll, c_void_p, c_ll)
bsf_jacobian_vjp = _fn("bsf_jacobian_vjp", c_int, bsf_t, c_void_p, c_ll, c_void_p, c_ll, c_void_p)
bsf_filter_backward_rows = _fn("bsf_filter_backward_rows", c_int, bsf_t, c_void_p, c_ll, c_void_p, c_int,
                               c_int, c_int, c_int, c_void_p, c_ll)
bsf_grad_frac_bits = _fn("bsf_grad_frac_bits", c_int, c_double)
bsf_grad_frac_bits_of = _fn("bsf_grad_frac_bits_of", c_int, bsf_t, c_double)
bsf_grad_absmax_rows = _fn("bsf_grad_absmax_rows", c_int, bsf_t, c_void_p, c_ll, c_int, c_int,
                           ctypes.POINTER(ctypes.c_float))
bsf_filter_host = _fn("bsf_filter_host", c_int, bsf_t, c_void_p, c_int, c_ll, c_void_p, c_int, c_void_p,
                      c_int, c_ll)
bsf_filter_two_pass = _fn("bsf_filter_two_pass", c_int, bsf_t, c_void_p, c_int, c_ll, c_void_p, c_int,
                          c_double, c_void_p, c_int, c_ll, ctypes.POINTER(ctypes.c_float))
bsf_grad_finalize = _fn("bsf_grad_finalize", c_int, bsf_t, c_void_p, c_ll, c_int, c_int, c_void_p, c_ll)
bsf_grad_halo_add = _fn("bsf_grad_halo_add", c_int, bsf_t, c_void_p, c_ll, c_void_p, c_ll, c_int)

class bsf_image_desc(ctypes.Structure):
    _fields_ = [("H", c_int), ("W", c_int), ("img", c_void_p), ("dtype", c_int), ("ld", c_ll),
                ("cov", c_void_p), ("out", c_void_p), ("out_dtype", c_int), ("ldo", c_ll)]


class bsf_batch_info_t(ctypes.Structure):
    _fields_ = [("B", c_int), ("frac_bits", c_int), ("arena_bytes", c_ll),
                ("scan_chunk", c_int * 4), ("blocks", c_int * 5), ("pixels", c_ll),
                ("graph_ready", c_int), ("persist_items", c_int), ("persist_grid", c_int),
                ("rows_per_item", c_int), ("stencil_tile_rows", c_int), ("persist_graph_ready", c_int),
                ("persist_groups", c_int)]


bsf_batch_t = ctypes.c_void_p
bsf_batch_create = _fn("bsf_batch_create", c_int, ctypes.POINTER(bsf_batch_t), c_int, c_int)
bsf_batch_destroy = _fn("bsf_batch_destroy", None, bsf_batch_t)
bsf_batch_set_stream = _fn("bsf_batch_set_stream", c_int, bsf_batch_t, c_void_p)
bsf_batch_stream = _fn("bsf_batch_stream", c_void_p, bsf_batch_t)
bsf_batch_set_precision = _fn("bsf_batch_set_precision", c_int, bsf_batch_t, c_int, c_double)
bsf_batch_set_tune_cache = _fn("bsf_batch_set_tune_cache", c_int, bsf_batch_t, ctypes.c_char_p)
bsf_batch_plan = _fn("bsf_batch_plan", c_int, bsf_batch_t, c_int, ctypes.POINTER(bsf_image_desc), c_int)
bsf_filter_batched = _fn("bsf_filter_batched", c_int, bsf_batch_t, c_int, ctypes.POINTER(bsf_image_desc), c_int)
bsf_batch_status = _fn("bsf_batch_status", c_int, bsf_batch_t)
bsf_batch_get_info = _fn("bsf_batch_get_info", c_int, bsf_batch_t, ctypes.POINTER(bsf_batch_info_t))
bsf_batch_last_error = _fn("bsf_batch_last_error", ctypes.c_char_p, bsf_batch_t)
bsf_batch_set_option = _fn("bsf_batch_set_option", c_int, bsf_batch_t, c_int, c_ll)

ERROR_NAMES = {v: k for k, v in _C.items() if k.startswith("BSF_E")}


class BsfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(h, rc: int) -> None:
    if rc != 0:
        msg = bsf_last_error(h).decode() if h else ""
        raise BsfError(rc, msg)


def declared_symbols(header: str = HEADER):
    """Names of the functions include/bsf.h declares."""
    with open(header) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsf_\w+)\s*\(", text)))


# --------------------------------------------------------------------------
# torch convenience wrapper
# --------------------------------------------------------------------------

_DTYPES = None


def _dtype_code(t) -> int:
    import torch
    global _DTYPES
    if _DTYPES is None:
        _DTYPES = {torch.uint8: BSF_U8, torch.float32: BSF_F32, torch.float64: BSF_F64}  # noqa: F821
    return _DTYPES[t.dtype]


_BOUNDARY = {"zero": 0, "replicate": 1, "symmetric": 2}


class BoxSplineFilter:
    """One library context for H x W images of order n on the current CUDA device.

    filter(img, cov, out_dtype) runs the whole forward pass on torch's current
    stream: step solve, extension + quantisation + running sums, finite
    differences.  img: [H][W] uint8/float32/float64 CUDA tensor; cov: [3][H][W]
    float32 CUDA tensor of cov_kind (0: C11, C12, C22; 1: log sigma, theta,
    log rho).  step_rule 2 (BSF_STEP_D2) selects the continuous-step filter,
    whose derivative with respect to cov comes from filter_jacobian.
    directions: BSF_DIRS_CARTESIAN (0), BSF_DIRS_SECOND (1: the box spline on
    (2,1), (1,2), (-1,2), (-2,1)) or BSF_DIRS_PAIR (2: both, switched per
    pixel by sector).
    memory_budget: bytes that box_spline_filter may keep from the forward for
    the backward beyond its inputs (None: no limit).  The continuous-step
    forward with a covariance that requires grad stores its Jacobian
    (12 bytes per pixel) only within the budget; above it the backward
    recomputes the running sums of the image and the Jacobian product
    (bsf_filter_backward) instead, with the same result bit for bit.
    """

    def __init__(self, H: int, W: int, n: int, boundary="symmetric", max_reach: int = -1,
                 precision: int = 1, frac_bits: int = -1, value_bound=None, step_rule: int = 0,
                 cov_kind: int = 0, directions: int = 0, memory_budget=None):
        if isinstance(boundary, str):
            boundary = _BOUNDARY[boundary]
        self.H, self.W, self.n = H, W, n
        self.cov_kind = cov_kind
        self.step_rule = step_rule
        self.memory_budget = memory_budget
        h = bsf_t()
        rc = bsf_create(ctypes.byref(h), H, W, 4, n, boundary, max_reach)
        if rc != 0:
            raise BsfError(rc, "bsf_create")
        self._h = h
        check(h, bsf_set_precision(h, precision, frac_bits))
        check(h, bsf_set_step_rule(h, step_rule))
        if value_bound is not None:
            check(h, bsf_set_value_bound(h, float(value_bound)))
        self.directions = 0
        if directions:
            self.set_option(BSF_OPT_DIRECTIONS, directions)  # noqa: F821

    def close(self):
        if getattr(self, "_h", None):
            bsf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _stream(self):
        import torch
        check(self._h, bsf_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def plan(self, cov):
        self._stream()
        assert cov.is_cuda and cov.dtype.is_floating_point and cov.is_contiguous()
        check(self._h, bsf_plan(self._h, ctypes.c_void_p(cov.data_ptr()), self.cov_kind))
        return self.info()

    def filter(self, img, cov, out=None, out_dtype=None):
        import torch
        self._stream()
        H, W = self.H, self.W
        assert img is None or (img.is_cuda and img.shape == (H, W) and img.stride(1) == 1)
        assert cov.is_cuda and cov.dtype == torch.float32 and cov.shape == (3, H, W) and cov.is_contiguous()
        if out is None:
            out = torch.empty((H, W), dtype=out_dtype or torch.float32, device=cov.device)
        oc = BSF_F32 if out.dtype == torch.float32 else BSF_F64  # noqa: F821
        if img is None:
            rc = bsf_filter(self._h, None, 0, W, ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                            ctypes.c_void_p(out.data_ptr()), oc, out.stride(0))
        else:
            rc = bsf_filter(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img), img.stride(0),
                            ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                            ctypes.c_void_p(out.data_ptr()), oc, out.stride(0))
        check(self._h, rc)
        return out

    def filter_two_pass(self, img, cov, frac: float = 0.5, out=None, want_sigma2: bool = False):
        """Algorithm 1: isotropic pass, then the residual pass (bsf_filter_two_pass).
        Returns out, or (out, sigma^2) with want_sigma2."""
        import torch
        self._stream()
        H, W = self.H, self.W
        assert img.is_cuda and img.shape == (H, W) and img.stride(1) == 1
        assert cov.is_cuda and cov.dtype == torch.float32 and cov.shape == (3, H, W) and cov.is_contiguous()
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=cov.device)
        oc = BSF_F32 if out.dtype == torch.float32 else BSF_F64  # noqa: F821
        s2 = ctypes.c_float()
        check(self._h, bsf_filter_two_pass(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img),
                                           img.stride(0), ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                                           float(frac), ctypes.c_void_p(out.data_ptr()), oc, out.stride(0),
                                           ctypes.byref(s2) if want_sigma2 else None))
        return (out, float(s2.value)) if want_sigma2 else out

    def filter_host(self, img, cov, out=None):
        """Forward filter from and to host (CPU) tensors, transfers overlapped
        with the work (bsf_filter_host); pinned tensors for the overlap."""
        import torch
        self._stream()
        H, W = self.H, self.W
        assert not img.is_cuda and img.shape == (H, W) and img.stride(1) == 1
        assert not cov.is_cuda and cov.dtype == torch.float32 and cov.shape == (3, H, W) and cov.is_contiguous()
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, pin_memory=True)
        assert not out.is_cuda and out.stride(1) == 1
        oc = BSF_F32 if out.dtype == torch.float32 else BSF_F64  # noqa: F821
        check(self._h, bsf_filter_host(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img),
                                       img.stride(0), ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                                       ctypes.c_void_p(out.data_ptr()), oc, out.stride(0)))
        return out

    def filter_jacobian(self, img, cov, out=None, jac=None):
        """Continuous-step forward and d out / d cov-plane: (out float32 [H][W], jac [3][H][W])."""
        import torch
        self._stream()
        H, W = self.H, self.W
        assert img.is_cuda and img.shape == (H, W) and img.stride(1) == 1
        assert cov.is_cuda and cov.dtype == torch.float32 and cov.shape == (3, H, W) and cov.is_contiguous()
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=cov.device)
        if jac is None:
            jac = torch.empty((3, H, W), dtype=torch.float32, device=cov.device)
        assert jac.is_contiguous() and out.dtype == torch.float32
        rc = bsf_filter_jacobian(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img),
                                 img.stride(0), ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                                 ctypes.c_void_p(out.data_ptr()), BSF_F32, out.stride(0),  # noqa: F821
                                 ctypes.c_void_p(jac.data_ptr()), W)
        check(self._h, rc)
        return out, jac

    def jacobian_vjp(self, gout, jac, gcov=None):
        """gcov[c] = gout * jac[c] (library kernel)."""
        import torch
        self._stream()
        H, W = self.H, self.W
        assert gout.is_cuda and gout.dtype == torch.float32 and gout.shape == (H, W) and gout.stride(1) == 1
        assert jac.is_contiguous() and jac.shape == (3, H, W)
        if gcov is None:
            gcov = torch.empty((3, H, W), dtype=torch.float32, device=gout.device)
        check(self._h, bsf_jacobian_vjp(self._h, ctypes.c_void_p(gout.data_ptr()), gout.stride(0),
                                        ctypes.c_void_p(jac.data_ptr()), W,
                                        ctypes.c_void_p(gcov.data_ptr())))
        return gcov

    def filter_rows(self, img, cov, y0: int, y1: int, out=None):
        """Rows [y0, y1) of the filtered image (float32), from the band's own running sums."""
        import torch
        self._stream()
        if out is None:
            out = torch.empty((y1 - y0, self.W), dtype=torch.float32, device=cov.device)
        rc = bsf_filter_rows(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img), img.stride(0),
                             ctypes.c_void_p(cov.data_ptr()), self.cov_kind, ctypes.c_void_p(out.data_ptr()),
                             BSF_F32 if out.dtype == torch.float32 else BSF_F64, out.stride(0), y0, y1)  # noqa: F821
        check(self._h, rc)
        return out

    def jacobian_bytes(self) -> int:
        """Bytes of the continuous-step Jacobian a stored-route forward keeps."""
        return 12 * self.H * self.W

    def stores_jacobian(self) -> bool:
        """True when the Jacobian fits memory_budget (the stored route)."""
        return self.memory_budget is None or self.jacobian_bytes() <= self.memory_budget

    def backward(self, gout, cov, gimg=None, want_gcov=False, want_gimg=True):
        """Gradients of the last filter: image gradient (D1; the covariance
        gradient of D1 is zero) or, for continuous steps, the image gradient
        and the covariance gradient, recomputed from the held running sums of
        the last pre-integrated image."""
        import torch
        self._stream()
        H, W = self.H, self.W
        assert gout.is_cuda and gout.dtype == torch.float32 and gout.shape == (H, W) and gout.stride(1) == 1
        if want_gimg and gimg is None:
            gimg = torch.empty((H, W), dtype=torch.float32, device=gout.device)
        gcov = torch.empty((3, H, W), dtype=torch.float32, device=gout.device) if want_gcov else None
        rc = bsf_filter_backward(self._h, ctypes.c_void_p(gout.data_ptr()), gout.stride(0),
                                 ctypes.c_void_p(cov.data_ptr()), self.cov_kind,
                                 ctypes.c_void_p(gimg.data_ptr()) if want_gimg else None,
                                 gimg.stride(0) if want_gimg else W,
                                 ctypes.c_void_p(gcov.data_ptr()) if want_gcov else None)
        check(self._h, rc)
        return gimg, gcov

    def grad_absmax_rows(self, gout, y0: int, y1: int) -> float:
        """max |gout| over rows [y0, y1) (library reduction; synchronises)."""
        self._stream()
        r = ctypes.c_float()
        check(self._h, bsf_grad_absmax_rows(self._h, ctypes.c_void_p(gout.data_ptr()), gout.stride(0),
                                            y0, y1, ctypes.byref(r)))
        return float(r.value)

    def grad_frac_bits(self, max_abs_gout: float) -> int:
        """The context's fraction-bit rule of the gradient weights (64- or 128-bit sums)."""
        return int(bsf_grad_frac_bits_of(self._h, float(max_abs_gout)))

    @staticmethod
    def _acc_ld(acc) -> int:
        # elements per row of an adjoint-sum tensor: int64 [rows][W], or int128
        # as int64 pairs [rows][W][2]
        return acc.stride(0) if acc.dim() == 2 else acc.stride(0) // 2

    def backward_rows(self, gout, cov, y0: int, y1: int, grad_bits: int):
        """Band adjoint: exact sums on image rows [a0, a1) = [y0 - R, y1 + R) clipped.

        Returns (acc, a0, a1), acc a CUDA tensor of int64 [a1 - a0][W] (64-bit
        adjoint sums) or of int64 pairs [a1 - a0][W][2] (int128, low word first:
        continuous steps and 128-bit contexts)."""
        import torch
        self._stream()
        inf = self.info()
        R = inf.R
        a0, a1 = max(0, y0 - R), min(self.H, y1 + R)
        shape = (a1 - a0, self.W) if inf.grad_elem_bytes == 8 else (a1 - a0, self.W, 2)
        acc = torch.empty(shape, dtype=torch.int64, device=gout.device)
        check(self._h, bsf_filter_backward_rows(self._h, ctypes.c_void_p(gout.data_ptr()), gout.stride(0),
                                                ctypes.c_void_p(cov.data_ptr()), self.cov_kind, y0, y1,
                                                grad_bits, ctypes.c_void_p(acc.data_ptr()), self._acc_ld(acc)))
        return acc, a0, a1

    def grad_finalize(self, acc, grad_bits: int, gimg=None):
        """gimg = RN32(acc) 2^-grad_bits (library kernel), float32 [rows][W]."""
        import torch
        self._stream()
        rows = acc.shape[0]
        if gimg is None:
            gimg = torch.empty((rows, self.W), dtype=torch.float32, device=acc.device)
        check(self._h, bsf_grad_finalize(self._h, ctypes.c_void_p(acc.data_ptr()), self._acc_ld(acc), rows,
                                         grad_bits, ctypes.c_void_p(gimg.data_ptr()), gimg.stride(0)))
        return gimg

    def grad_halo_add(self, acc, halo):
        """acc += halo modulo 2^64 or 2^128 (library kernel): CUDA tensors of the
        same shape, int64 [rows][W] or int64 pairs [rows][W][2] (acc may be a row
        slice of a larger tensor)."""
        import torch
        self._stream()
        assert acc.dtype == torch.int64 and halo.dtype == torch.int64 and acc.shape == halo.shape
        assert acc.is_cuda and halo.is_cuda and acc.stride(-1) == 1 and (acc.dim() == 2 or acc.stride(1) == 2)
        halo = halo.to(acc.device).contiguous()
        check(self._h, bsf_grad_halo_add(self._h, ctypes.c_void_p(acc.data_ptr()), self._acc_ld(acc),
                                         ctypes.c_void_p(halo.data_ptr()), self._acc_ld(halo), acc.shape[0]))
        return acc

    def preintegrate(self, img):
        self._stream()
        check(self._h, bsf_preintegrate(self._h, ctypes.c_void_p(img.data_ptr()), _dtype_code(img),
                                        img.stride(0)))

    def set_option(self, option: int, value: int):
        check(self._h, bsf_set_option(self._h, option, value))
        if option == BSF_OPT_DIRECTIONS:  # noqa: F821
            self.directions = int(value)

    def set_profiling(self, on: bool = True):
        check(self._h, bsf_set_profiling(self._h, 1 if on else 0))

    def read_profile(self):
        """{phase name: (total ms, executions)} since the last read (syncs)."""
        n = BSF_NUM_PHASES  # noqa: F821
        ms = (c_double * n)()
        cnt = (c_int * n)()
        rc = bsf_read_profile(self._h, ms, cnt)
        if rc < 0:
            check(self._h, rc)
        names = ["steps", "rows", "d3", "d2", "d4", "stencil", "bwd_scatter", "bwd_scans", "bwd_fold",
                 "second", "tiles", "vjp"]
        return {names[i]: (ms[i], cnt[i]) for i in range(n)}

    def status(self) -> int:
        return bsf_status(self._h)

    def info(self) -> bsf_info_t:
        inf = bsf_info_t()
        check(self._h, bsf_get_info(self._h, ctypes.byref(inf)))
        return inf

    def steps(self):
        import torch
        dst = torch.empty((4, self.H, self.W), dtype=torch.int16, device="cuda")
        self._stream()
        check(self._h, bsf_copy_steps(self._h, ctypes.c_void_p(dst.data_ptr())))
        return dst.view(torch.uint16) if hasattr(torch, "uint16") else dst

    def preintegrated(self):
        import torch
        inf = self.info()
        nb = inf.Hp * inf.Wp * inf.elem_bytes
        if self.directions == BSF_DIRS_PAIR:  # noqa: F821  (the second set's sums follow)
            nb *= 2
        dst = torch.empty(nb, dtype=torch.uint8, device="cuda")
        self._stream()
        check(self._h, bsf_copy_preintegrated(self._h, ctypes.c_void_p(dst.data_ptr())))
        return dst, inf


def _make_autograd():
    import torch

    class BoxSplineFilterFunction(torch.autograd.Function):
        """out = filter(img, cov).  Integer steps (D1): backward gives d/dimg
        through the library's adjoint kernels (the steps are piecewise
        constant, so d/dcov = 0).  Continuous steps (D2): when cov requires
        grad and the Jacobian (12 bytes per pixel) fits the filter's
        memory_budget, the forward also writes d out / d cov-plane and the
        backward multiplies it by the incoming gradient (library kernel);
        above the budget the forward keeps nothing but its inputs and the
        backward recomputes the image's running sums and the Jacobian product
        (bsf_preintegrate, bsf_filter_backward).  The image gradient of D2
        (uint128 contexts) comes from the library's adjoint kernels."""

        @staticmethod
        def forward(ctx, img, cov, filt):
            ctx.filt = filt
            ctx.d2 = filt.step_rule == BSF_STEP_D2  # noqa: F821
            ctx.recompute = False
            if ctx.d2:
                cov = cov.contiguous()
                img = img.contiguous()
                if cov.requires_grad and filt.stores_jacobian():
                    out, jac = filt.filter_jacobian(img, cov)
                    ctx.save_for_backward(img, cov, jac)
                    return out
                ctx.recompute = cov.requires_grad
                ctx.save_for_backward(img, cov)
                return filt.filter(img, cov)
            out = filt.filter(img.contiguous(), cov.contiguous())
            ctx.save_for_backward(cov)
            return out

        @staticmethod
        def backward(ctx, gout):
            gout = gout.contiguous().float()
            if ctx.d2:
                saved = ctx.saved_tensors
                img, cov = saved[0], saved[1]
                gimg = gcov = None
                if ctx.recompute:
                    # the running sums of this image again (another call may
                    # have replaced them), then both gradients from them
                    ctx.filt.preintegrate(img)
                    gimg, gcov = ctx.filt.backward(gout, cov, want_gimg=ctx.needs_input_grad[0],
                                                   want_gcov=ctx.needs_input_grad[1])
                    return gimg, gcov, None
                if ctx.needs_input_grad[0]:
                    gimg, _ = ctx.filt.backward(gout, cov, want_gimg=True, want_gcov=False)
                if ctx.needs_input_grad[1]:
                    gcov = ctx.filt.jacobian_vjp(gout, saved[2])
                return gimg, gcov, None
            (cov,) = ctx.saved_tensors
            gimg, gcov = ctx.filt.backward(gout.contiguous().float(), cov,
                                           want_gcov=ctx.needs_input_grad[1])
            return gimg, gcov, None

    return BoxSplineFilterFunction


def box_spline_filter(img, cov, filt: "BoxSplineFilter"):
    """Differentiable forward filter (torch.autograd) through the library."""
    global _AUTOGRAD
    try:
        fn = _AUTOGRAD
    except NameError:
        fn = _AUTOGRAD = _make_autograd()
    return fn.apply(img, cov, filt)


class BatchFilter:
    """A batch of images of uneven sizes on one device arena (bsf_batch_*).

    imgs / covs / outs are lists of CUDA tensors ([H][W], [3][H][W] float32,
    [H][W]).  The batch runs on its own stream; ``stream()`` gives it as a
    torch external stream for ordering with torch work.
    """

    def __init__(self, n: int, boundary="symmetric", frac_bits: int = -1, value_bound: float = 0.0):
        if isinstance(boundary, str):
            boundary = _BOUNDARY[boundary]
        b = bsf_batch_t()
        rc = bsf_batch_create(ctypes.byref(b), n, boundary)
        if rc != 0:
            raise BsfError(rc, "bsf_batch_create")
        self._b = b
        self._chk(bsf_batch_set_precision(b, frac_bits, float(value_bound)))

    def _chk(self, rc):
        if rc != 0:
            raise BsfError(rc, bsf_batch_last_error(self._b).decode())

    def close(self):
        if getattr(self, "_b", None):
            bsf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tune_cache(self, path: str):
        self._chk(bsf_batch_set_tune_cache(self._b, path.encode()))

    def plan(self, imgs, covs, outs, autotune: bool = False):
        B = len(imgs)
        arr = (bsf_image_desc * B)()
        for i, (im, cv, ot) in enumerate(zip(imgs, covs, outs)):
            H, W = im.shape
            assert im.is_cuda and im.stride(1) == 1 and ot.is_cuda and ot.shape == (H, W) and ot.stride(1) == 1
            assert cv.is_cuda and cv.dtype.itemsize == 4 and cv.shape == (3, H, W) and cv.is_contiguous()
            arr[i] = bsf_image_desc(H, W, im.data_ptr(), _dtype_code(im), im.stride(0), cv.data_ptr(),
                                    ot.data_ptr(), BSF_F32 if ot.dtype.itemsize == 4 else BSF_F64,  # noqa: F821
                                    ot.stride(0))
        self._descs = arr
        self._B = B
        self._chk(bsf_batch_plan(self._b, B, arr, BSF_BATCH_AUTOTUNE if autotune else 0))  # noqa: F821
        return self.info()

    def run(self, flags: int = 0):
        self._chk(bsf_filter_batched(self._b, self._B, self._descs, flags))

    def set_option(self, option: int, value: int):
        self._chk(bsf_batch_set_option(self._b, option, int(value)))

    def status(self) -> int:
        return bsf_batch_status(self._b)

    def info(self) -> bsf_batch_info_t:
        inf = bsf_batch_info_t()
        self._chk(bsf_batch_get_info(self._b, ctypes.byref(inf)))
        return inf

    def stream(self):
        import torch
        return torch.cuda.ExternalStream(bsf_batch_stream(self._b))
