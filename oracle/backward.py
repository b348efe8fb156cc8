"""Adjoint of the D1 filter with respect to the image.

Oracle module (test infrastructure only; see the package docstring).

The forward filter is linear in the image:  out(p) = sum_j K_p(j) f~(p + j) / D_p
with f~ the extended image (kernels.py).  For a loss gradient gout = dL/dout
the image gradient is the transposed operator

    gimg(i) = sum_{r : ext(r) = i} sum_p gout(p) K_p(r - p) / D_p,

a scatter of every output pixel's kernel followed by the adjoint of the
boundary extension (every padded position adds back onto the image pixel it
copies).  The paper has no backward pass; this is the adjoint of its
BoxFilter algorithm (Section 1.1).

Number format (reading; the forward's fixed point carried over): each output
pixel's weight gout(p)/D_p is quantised once,

    g(p) = round-half-even( RN32( RN32(gout(p) 2^qg) / RN32(D_p) ) ),

computed in float32 (gout(p) 2^qg is exact), and everything after that is
exact integer arithmetic; the result is RN32(acc) 2^-qg.  qg is chosen from
max |gout| so that the exact gradient keeps 2^8 of headroom in 62 bits:
qg = 54 - ceil(log2 max|gout|), clamped to [0, 100].

Contexts whose running sums are 128 bits wide (masses beyond 2^64) take
the same number format in 128 bits: qg = 118 - ceil(log2 max|gout|) in
[0, 126], exact sums modulo 2^128 (adjoint_direct_wide).

Two routes, pinned against each other:
  adjoint_direct   -- the definition: explicit kernels, explicit scatter;
  adjoint_modular  -- the pipeline's transpose: scatter w_t g(p) at the taps,
                      then reversed n-fold running sums (suffix sums) along
                      d4, d2, d3, d1, then the extension adjoint, all mod 2^64.
"""
from __future__ import annotations

import math

import numpy as np

from . import modular
from .kernels import extend_index, kernel_d1, kernel_mass
from .rounding import rn_f32_int

U64 = np.uint64


def grad_frac_bits(max_abs_gout: float) -> int:
    """qg = 54 - ceil(log2 m) for m = max |gout| (float32), clamped to [0, 100]."""
    m = float(np.float32(max_abs_gout))
    if m == 0.0 or not math.isfinite(m):
        c = 0
    else:
        mant, e = math.frexp(m)          # m = mant 2^e, mant in [0.5, 1)
        c = e - 1 if mant == 0.5 else e  # ceil(log2 m)
    return int(min(max(54 - c, 0), 100))


def quantize_weights(gout: np.ndarray, D: np.ndarray, qg: int) -> np.ndarray:
    """g(p) = RNE(RN32(gout 2^qg) / RN32(D)) as int64, computed in float32."""
    x = gout.astype(np.float32) * np.float32(math.ldexp(1.0, qg))
    Dobj = np.asarray(D).astype(object)
    y = np.vectorize(rn_f32_int, otypes=[np.float32])(Dobj)
    g = (x / y).astype(np.float32)
    return np.rint(g).astype(np.int64)


def _finish(acc, qg: int) -> np.ndarray:
    acc = np.asarray(acc, dtype=object)
    v = np.vectorize(rn_f32_int, otypes=[np.float32])(acc)
    return (v * np.float32(math.ldexp(1.0, -qg))).astype(np.float32)


def adjoint_direct_acc(g: np.ndarray, Lfield: np.ndarray, n: int, boundary: int) -> np.ndarray:
    """Exact integer gradient accumulator: sum_p g(p) K_p(r - p), folded onto the image."""
    H, W = g.shape
    acc = np.zeros((H, W), dtype=object)
    for y in range(H):
        for x in range(W):
            gv = int(g[y, x])
            if gv == 0:
                continue
            K, ox, oy = kernel_d1(tuple(int(Lfield[k, y, x]) for k in range(4)), n)
            kh, kw = K.shape
            yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
            xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
            for a in range(kh):
                if not yv[a]:
                    continue
                row = K[a]
                for b in range(kw):
                    if xv[b] and row[b] != 0:
                        acc[yi[a], xi[b]] += gv * int(row[b])
    return acc


def adjoint_direct(gout: np.ndarray, Lfield: np.ndarray, n: int, boundary: int, qg: int):
    D = modular.masses(Lfield, n)
    g = quantize_weights(gout, D, qg)
    return _finish(adjoint_direct_acc(g, Lfield, n, boundary), qg)


# ---------------------------------------------------------------------------
# 128-bit number format (contexts whose kernel masses exceed the reach of
# 64-bit weights): the same route with qg = 118 - ceil(log2 max|gout|) in
# [0, 126], exact sums modulo 2^128 (Python integers here, no modulus needed)
# ---------------------------------------------------------------------------

def grad_frac_bits_wide(max_abs_gout: float) -> int:
    """qg = 118 - ceil(log2 m) for m = max |gout| (float32), clamped to [0, 126]."""
    m = float(np.float32(max_abs_gout))
    if m == 0.0 or not math.isfinite(m):
        c = 0
    else:
        mant, e = math.frexp(m)
        c = e - 1 if mant == 0.5 else e
    return int(min(max(118 - c, 0), 126))


def quantize_weights_wide(gout: np.ndarray, D: np.ndarray, qg: int) -> np.ndarray:
    """g(p) = RNE(RN32(gout 2^qg) / RN32(D)) as Python integers (object array)."""
    x = gout.astype(np.float32) * np.float32(math.ldexp(1.0, qg))
    Dobj = np.asarray(D).astype(object)
    y = np.vectorize(rn_f32_int, otypes=[np.float32])(Dobj)
    g = (x / y).astype(np.float32)
    return np.vectorize(lambda v: int(round(float(v))), otypes=[object])(g)


def adjoint_direct_wide(gout: np.ndarray, Lfield: np.ndarray, n: int, boundary: int):
    """The image gradient in the 128-bit number format, by the definition."""
    qg = grad_frac_bits_wide(float(np.abs(gout).max(initial=0.0)))
    g = quantize_weights_wide(gout, modular.masses(Lfield, n), qg)
    return _finish(adjoint_direct_acc(g, Lfield, n, boundary), qg)


def _suffix64(G: np.ndarray, k: int) -> None:
    """One inclusive suffix sum of G (uint64, in place) along direction d_k:
    G(x) <- G(x) + G(x + d_k), zero past the end of the domain."""
    Hp, Wp = G.shape
    if k == 0:
        G[:, :] = np.flip(np.cumsum(np.flip(G, axis=1), axis=1, dtype=U64), axis=1)
    elif k == 2:
        G[:, :] = np.flip(np.cumsum(np.flip(G, axis=0), axis=0, dtype=U64), axis=0)
    elif k == 1:      # d2 = (1, 1): G(x, y) += G(x+1, y+1)
        for y in range(Hp - 2, -1, -1):
            G[y, :-1] += G[y + 1, 1:]
    elif k == 3:      # d4 = (-1, 1): G(x, y) += G(x-1, y+1)
        for y in range(Hp - 2, -1, -1):
            G[y, 1:] += G[y + 1, :-1]


def adjoint_modular_acc(g: np.ndarray, Lfield: np.ndarray, n: int, boundary: int, R: int):
    """Transpose of the running-sum pipeline applied to integer weights g,
    mod 2^64, returned as signed int64 image accumulators."""
    H, W = g.shape
    Hp, Wp = H + 2 * R, W + 2 * R
    G = np.zeros((Hp, Wp), dtype=U64)
    yy, xx = np.mgrid[0:H, 0:W]
    L = Lfield.astype(np.int64)
    c = (n * (L - 1)) // 2
    base_x = xx + R + c[0] + c[1] - c[3]
    base_y = yy + R + c[1] + c[2] + c[3]
    gu = g.astype(np.int64).view(U64)
    with np.errstate(over="ignore"):
        for t, w in modular.tap_weights(n):
            tx = base_x - t[0] * L[0] - t[1] * L[1] + t[3] * L[3]
            ty = base_y - t[1] * L[1] - t[2] * L[2] - t[3] * L[3]
            contrib = (U64(w % (1 << 64)) * gu)
            np.add.at(G, (ty.ravel(), tx.ravel()), contrib.ravel())
        for k in reversed(modular.SCAN_ORDER):   # d4, d2, d3, d1
            for _ in range(n):
                _suffix64(G, k)
        # adjoint of the extension: every padded position adds onto its source
        yi, yv = extend_index(np.arange(-R, H + R), H, boundary)
        xi, xv = extend_index(np.arange(-R, W + R), W, boundary)
        acc = np.zeros((H, W), dtype=U64)
        rows = np.where(yv)[0]
        cols = np.where(xv)[0]
        sub = G[np.ix_(rows, cols)]
        np.add.at(acc, (np.repeat(yi[rows], len(cols)), np.tile(xi[cols], len(rows))), sub.ravel())
    return acc.view(np.int64)


def adjoint_modular(gout: np.ndarray, Lfield: np.ndarray, n: int, boundary: int, qg: int, R: int):
    D = modular.masses(Lfield, n)
    g = quantize_weights(gout, D, qg)
    return _finish(adjoint_modular_acc(g, Lfield, n, boundary, R), qg)


def adjoint_f64(gout: np.ndarray, Lfield: np.ndarray, n: int, boundary: int) -> np.ndarray:
    """The exact adjoint in float64 (no quantisation): sum_p gout(p) K_p(r-p) / D_p folded."""
    H, W = gout.shape
    acc = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            Lt = tuple(int(Lfield[k, y, x]) for k in range(4))
            K, ox, oy = kernel_d1(Lt, n)
            wgt = float(gout[y, x]) / float(kernel_mass(Lt, n))
            kh, kw = K.shape
            yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
            xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
            Kf = K.astype(np.float64) * wgt
            m = np.outer(yv, xv)
            np.add.at(acc, (np.repeat(yi, kw).reshape(kh, kw)[m], np.tile(xi, kh).reshape(kh, kw)[m]), Kf[m])
    return acc
