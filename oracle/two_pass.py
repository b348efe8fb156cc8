"""Algorithm 1: an isotropic pass, then the space-variant residual pass.

Oracle module (test infrastructure only; see the package docstring).

The paper splits the target covariance C = sigma^2 I + Delta C (eq.
"SigmaIso"): the image is first filtered with the isotropic box spline of
covariance sigma^2 I, then with the space-variant box spline of the residual
Delta C = C - sigma^2 I; by Proposition 1 the covariances add, and by
Proposition 2 (the split) the two filters compose into one of covariance C.
Delta C must stay within the elongation bound, which gives eq. "condition2"
on sigma^2; sigma^2 is set to half that bound (Algorithm 1, step 1).

Readings: one global sigma^2 (the first pass of Algorithm 1 is the
space-invariant BoxFilter): half the smallest condition-2 bound over
the field (floored at zero); the bound is written algebraically,
    root = sqrt((C11 - C22)^2 + 4 C12^2),
    tan(phi) = ((C22 - C11) + root) / (2 C12) if C22 >= C11,
               2 C12 / ((C11 - C22) + root) otherwise  (phi: orientation of C),
    t = |tan(phi) - 1/tan(phi)| / 2,
    (e + 1)/(e - 1) = (1 + t) / sqrt(1 + t^2)  (e = e(phi) of eq. "boundE"),
                    = (1 + 1/t) / sqrt(1 + 1/t^2) for t > 1,
    bound = (C11 + C22 - (1 + t)/sqrt(1 + t^2) root) / 2,
with the factor 1 on the axes (C12 = 0, e infinite), evaluated in float64 in
this order.  Both passes use the integer-step filter (D1) with one q, and the
first pass's output is the second pass's input as the float32 image the
output rule produces.
"""
from __future__ import annotations

import math

import numpy as np

from . import modular

_F = np.float32


def condition2_bound(C11, C12, C22) -> float:
    """Right side of eq. "condition2", algebraic form (float64, fixed order).

    Pinned by tests against params.condition2_bound (trigonometric form)."""
    c11, c12, c22 = float(C11), float(C12), float(C22)
    d = c11 - c22
    root = math.sqrt(d * d + 4.0 * (c12 * c12))
    if c12 == 0.0:
        ratio = 1.0
    else:
        # tan(phi) = (lambda_max - C11) / C12 = C12 / (lambda_max - C22), in the
        # form without cancellation
        tn = ((c22 - c11) + root) / (2.0 * c12) if c22 >= c11 else (2.0 * c12) / ((c11 - c22) + root)
        t = abs(tn - 1.0 / tn) / 2.0
        if t > 1.0:
            u = 1.0 / t
            ratio = (1.0 + u) / math.sqrt(1.0 + u * u)
        else:
            ratio = (1.0 + t) / math.sqrt(1.0 + t * t)
    return ((c11 + c22) - ratio * root) / 2.0


def sigma2_global(cov: np.ndarray, frac: float = 0.5) -> np.float32:
    """sigma^2 = frac * min over pixels of max(bound, 0), rounded to float32."""
    m = math.inf
    for c11, c12, c22 in zip(cov[0].ravel(), cov[1].ravel(), cov[2].ravel()):
        m = min(m, max(condition2_bound(c11, c12, c22), 0.0))
    return _F(frac * m)


def split_field(cov: np.ndarray, sigma2):
    """(isotropic field sigma^2 I, residual field C - sigma^2 I), float32 [3][H][W]."""
    s = _F(sigma2)
    iso = np.empty_like(cov, dtype=_F)
    iso[0] = s
    iso[1] = 0
    iso[2] = s
    res = np.stack([(cov[0] - s).astype(_F), cov[1].astype(_F), (cov[2] - s).astype(_F)])
    return iso, np.ascontiguousarray(res)


def algorithm1(f: np.ndarray, cov: np.ndarray, n: int, boundary: int, q: int, R: int,
               bits: int = 64, frac: float = 0.5, out_dtype=np.float32):
    """Both passes of Algorithm 1 through the running-sum pipeline of
    modular.filter_modular (same R and q in both).  Returns (out, sigma2, g)."""
    s2 = sigma2_global(cov, frac)
    iso, res = split_field(cov, s2)
    g = modular.filter_modular(f, iso, n, boundary, q=q, bits=bits, out_dtype=np.float32, R=R)
    out = modular.filter_modular(g, res, n, boundary, q=q, bits=bits, out_dtype=out_dtype, R=R)
    return out, s2, g
