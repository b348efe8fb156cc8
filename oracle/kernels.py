"""Discrete box-spline kernels and the direct (definition) filter.

Oracle module (test infrastructure only; see the package docstring).

What the pre-integration + finite-difference pipeline computes (Section 1.1,
the BoxFilter algorithm) is, in exact arithmetic, a space-variant discrete
correlation

    out(p) = sum_j K_p(j) f~(p + j) / mass(K_p),

where K_p is the 2-D convolution of N = 4 one-dimensional kernels, the k-th
living on the line Z d_k.  With integer steps L_k (the D1 rule) the k-th
kernel is the n-fold convolution of L_k unit samples (a discrete box of L_k
taps, n times), centred; its mass is L_k^n.  This module builds K_p from that
definition and correlates directly: no running sums anywhere.

f~ is the image extended beyond its borders by one of three rules (the paper
is silent on borders; this is a reading): zero, replicate (clamp), or
symmetric half-sample (d c b a | a b c d).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .params import DIRS

ZERO, REPLICATE, SYMMETRIC = 0, 1, 2
BOUNDARY_NAMES = {"zero": ZERO, "replicate": REPLICATE, "symmetric": SYMMETRIC}


def extend_index(i, N: int, boundary: int):
    """Map integer coordinates i (array) into [0, N) by the extension rule.

    Returns (index, valid): valid is False where the zero rule applies.
    """
    i = np.asarray(i, dtype=np.int64)
    if boundary == ZERO:
        valid = (i >= 0) & (i < N)
        return np.clip(i, 0, N - 1), valid
    if boundary == REPLICATE:
        return np.clip(i, 0, N - 1), np.ones(i.shape, dtype=bool)
    if boundary == SYMMETRIC:
        m = np.mod(i, 2 * N)
        m = np.where(m >= N, 2 * N - 1 - m, m)
        return m, np.ones(i.shape, dtype=bool)
    raise ValueError(boundary)


def extend_image(f: np.ndarray, pad: int, boundary: int) -> np.ndarray:
    """f~ on [-pad, W+pad) x [-pad, H+pad), as an array (object dtype kept)."""
    H, W = f.shape
    yi, yv = extend_index(np.arange(-pad, H + pad), H, boundary)
    xi, xv = extend_index(np.arange(-pad, W + pad), W, boundary)
    out = f[np.ix_(yi, xi)].copy()
    mask = np.outer(yv, xv)
    if f.dtype == object:
        out[~mask] = 0
    else:
        out[~mask] = 0
    return out


@lru_cache(maxsize=None)
def box_power_1d(L: int, n: int) -> tuple:
    """Integer weights of the n-fold convolution of L unit samples (length n(L-1)+1).

    Its mass is L^n and it is symmetric; offsets run from -n(L-1)/2 to
    n(L-1)/2 (an integer for admissible L).
    """
    h = np.ones(1, dtype=object)
    box = np.ones(L, dtype=object)
    for _ in range(n):
        h = np.convolve(h, box)
    return tuple(int(v) for v in h)


@lru_cache(maxsize=4096)
def kernel_d1(L: tuple, n: int, dirs: tuple = DIRS):
    """2-D integer kernel K for integer steps L = (L1..L4), order n.

    Returns (K, ox, oy): K[oy + dy, ox + dx] is the weight at offset (dx, dy)
    (dx the column offset).  Built as the convolution of the four line
    kernels box_power_1d(L_k, n) placed on Z d_k, each centred.  Entries are
    Python ints (object array); sum(K) = prod_k L_k^n.  dirs: the grid
    vectors d_k (default the Cartesian set; the second set of Section 2.3 is
    ((2,1), (1,2), (-1,2), (-2,1))).
    """
    K = np.ones((1, 1), dtype=object)
    ox = oy = 0
    for k, (dx, dy) in enumerate(dirs):
        h = box_power_1d(int(L[k]), n)
        half = n * (int(L[k]) - 1) // 2
        offs = np.arange(-half, half + 1)
        sx = offs * dx
        sy = offs * dy
        nx0, nx1 = -ox + sx.min(), K.shape[1] - 1 - ox + sx.max()
        ny0, ny1 = -oy + sy.min(), K.shape[0] - 1 - oy + sy.max()
        Kn = np.zeros((ny1 - ny0 + 1, nx1 - nx0 + 1), dtype=object)
        nox, noy = -nx0, -ny0
        for w, ddx, ddy in zip(h, sx, sy):
            y0 = noy - oy + ddy
            x0 = nox - ox + ddx
            Kn[y0:y0 + K.shape[0], x0:x0 + K.shape[1]] += w * K
        K, ox, oy = Kn, nox, noy
    return K, ox, oy


def kernel_mass(L, n: int) -> int:
    m = 1
    for v in L:
        m *= int(v) ** n
    return m


def correlate_exact(fq: np.ndarray, Lfield: np.ndarray, n: int, boundary: int,
                    pixels=None, dirs: tuple = DIRS):
    """Exact integer accumulator acc(p) = sum_j K_p(j) fq~(p + j) (Python ints).

    fq is an integer image (int64 or object), Lfield is int[4][H][W].
    ``pixels`` is an optional iterable of (y, x); default all pixels.
    Returns a dict {(y, x): acc} when pixels is given, else an object array.
    """
    H, W = fq.shape
    fobj = fq.astype(object)
    out = {} if pixels is not None else np.empty((H, W), dtype=object)
    it = pixels if pixels is not None else ((y, x) for y in range(H) for x in range(W))
    for (y, x) in it:
        Lt = tuple(int(Lfield[k, y, x]) for k in range(4))
        K, ox, oy = kernel_d1(Lt, n, dirs)
        kh, kw = K.shape
        yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
        xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
        patch = fobj[np.ix_(yi, xi)]
        patch = np.where(np.outer(yv, xv), patch, 0)
        acc = int((K * patch).sum())
        out[(y, x)] = acc
    return out


def correlate_f64(f: np.ndarray, Lfield: np.ndarray, n: int, boundary: int, pixels=None):
    """Float64 direct filter out(p) = sum_j K_p(j) f~(p+j) / mass, no quantisation.

    Each product K(j) f(p+j) is rounded once to float64 and the products are
    summed with math.fsum (correctly rounded), so the result is within a few
    units in the last place of the exact value.  Returns a float64 array, or
    a dict when ``pixels`` is given.
    """
    import math
    H, W = f.shape
    out = {} if pixels is not None else np.empty((H, W), dtype=np.float64)
    it = pixels if pixels is not None else ((y, x) for y in range(H) for x in range(W))
    for (y, x) in it:
        Lt = tuple(int(Lfield[k, y, x]) for k in range(4))
        K, ox, oy = kernel_d1(Lt, n)
        kh, kw = K.shape
        yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
        xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
        patch = f[np.ix_(yi, xi)].astype(np.float64)
        mask = np.outer(yv, xv)
        Kf = K.astype(np.float64)
        terms = (Kf * patch)[mask & (K != 0)]
        val = math.fsum(terms.tolist()) / float(kernel_mass(Lt, n))
        out[(y, x)] = val
    return out


def kernel_d1_int64(L: tuple, n: int):
    """kernel_d1 built with int64 arithmetic (scipy.signal.convolve2d of the
    four line kernels); exact while the mass prod L^n stays below 2^62.
    Returns (K, ox, oy) like kernel_d1.  Pinned by tests against kernel_d1."""
    from scipy.signal import convolve2d
    if kernel_mass(L, n) >= (1 << 62):
        raise OverflowError("kernel mass too large for int64")
    K = np.ones((1, 1), dtype=np.int64)
    for k, (dx, dy) in enumerate(DIRS):
        h = np.array(box_power_1d(int(L[k]), n), dtype=np.int64)
        m = len(h)
        if (dx, dy) == (1, 0):
            line = h.reshape(1, m)
        elif (dx, dy) == (0, 1):
            line = h.reshape(m, 1)
        elif (dx, dy) == (1, 1):
            line = np.diag(h)
        else:  # (-1, 1): x decreases as y increases
            line = np.fliplr(np.diag(h))
        K = convolve2d(K, line)
    oy, ox = (K.shape[0] - 1) // 2, (K.shape[1] - 1) // 2
    return K, ox, oy


def correlate_exact_sampled(fq: np.ndarray, Lfield: np.ndarray, n: int, boundary: int, pixels):
    """Exact accumulators at sampled pixels for small-valued integer images
    (|fq| < 2^24), with int64 kernels split into 31-bit limbs so every dot
    product is exact in int64.  Returns {(y, x): Python int}."""
    H, W = fq.shape
    f64 = fq.astype(np.int64)
    cache = {}
    out = {}
    for (y, x) in pixels:
        Lt = tuple(int(Lfield[k, y, x]) for k in range(4))
        if Lt not in cache:
            K, ox, oy = kernel_d1_int64(Lt, n)
            cache[Lt] = (K >> 31, K & ((1 << 31) - 1), ox, oy)
        Khi, Klo, ox, oy = cache[Lt]
        kh, kw = Khi.shape
        yi, yv = extend_index(np.arange(y - oy, y - oy + kh), H, boundary)
        xi, xv = extend_index(np.arange(x - ox, x - ox + kw), W, boundary)
        patch = np.where(np.outer(yv, xv), f64[np.ix_(yi, xi)], 0)
        out[(y, x)] = (int((Khi * patch).sum()) << 31) + int((Klo * patch).sum())
    return out
