"""The paper's pipeline -- pre-integration, then per-pixel finite differences --
run plainly and sequentially in exact two's-complement modular arithmetic.

Oracle module (test infrastructure only; see the package docstring).

Pre-integration (Section 1.1, the running sum; Algorithm 3, step 2, gives the
same recursions for the other direction set): for each direction d_k, n times,

    S(x) <- S(x) + S(x - d_k)        (S = 0 before the start of the domain)

over the padded domain P = [-R, W+R) x [-R, H+R), starting from the extended
quantised image.  The step-length factor of the paper's recursion (sqrt(5)
there, sqrt(2) on the diagonals here) is left out: the normalisation is done
once, in grid-step units, at the end.  Directions are scanned in the order
d1, d3, d2, d4.

Finite differences (Section 1.1, the 16-tap mesh, generalised to order n):

    acc(p) = sum_t w_t S(p + sum_k (c_k - t_k L_k) d_k),
    w_t = prod_k (-1)^t_k C(n, t_k),  c_k = n (L_k - 1)/2,  t in {0..n}^4,

evaluated mod 2^b and read back as a signed integer.  Whenever the true
accumulator satisfies |acc| < 2^(b-1) the wrap-around of the running sums
cancels exactly, so acc equals the direct correlation of kernels.py.

b = 64 uses numpy uint64 (whose arithmetic wraps mod 2^64); b = 128 uses a
pair of uint64 limbs (lo, hi) with explicit carries.
Pinned by tests: equals kernels.correlate_exact bit for bit on integer images
(all n <= 3 and all borders), and equals a pure-Python big-integer running
sum on tiny inputs.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

from . import params
from .kernels import extend_image, kernel_mass
from .rounding import quantize, finalize

U64 = np.uint64
MASK64 = (1 << 64) - 1


# ----------------------------- 128-bit limbs -------------------------------

class U128:
    """Array of unsigned 128-bit integers as two uint64 limbs."""

    __slots__ = ("lo", "hi")

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, dtype=U64)
        self.hi = np.asarray(hi, dtype=U64)

    @staticmethod
    def from_ints(a: np.ndarray) -> "U128":
        a = np.asarray(a, dtype=object)
        m = np.vectorize(lambda v: int(v) & ((1 << 128) - 1), otypes=[object])(a)
        lo = np.vectorize(lambda v: v & MASK64, otypes=[object])(m).astype(U64)
        hi = np.vectorize(lambda v: v >> 64, otypes=[object])(m).astype(U64)
        return U128(lo, hi)

    def copy(self):
        return U128(self.lo.copy(), self.hi.copy())

    def __getitem__(self, idx):
        return U128(self.lo[idx], self.hi[idx])

    def __setitem__(self, idx, v: "U128"):
        self.lo[idx] = v.lo
        self.hi[idx] = v.hi

    def __add__(self, o: "U128") -> "U128":
        lo = self.lo + o.lo
        c = (lo < self.lo).astype(U64)
        return U128(lo, self.hi + o.hi + c)

    def __sub__(self, o: "U128") -> "U128":
        lo = self.lo - o.lo
        bo = (self.lo < o.lo).astype(U64)
        return U128(lo, self.hi - o.hi - bo)

    def to_signed_ints(self) -> np.ndarray:
        lo = self.lo.astype(object)
        hi = self.hi.astype(object)
        v = lo + (hi << 64)
        return np.vectorize(lambda t: t - (1 << 128) if t >> 127 else t, otypes=[object])(v)


def _zeros_like_u128(shape):
    return U128(np.zeros(shape, U64), np.zeros(shape, U64))


# ------------------------------ scans --------------------------------------

def _scan64(S: np.ndarray, k: int) -> None:
    """One inclusive running sum of S (uint64, in place) along direction d_k."""
    Hp, Wp = S.shape
    if k == 0:      # d1 = (1, 0): along each row
        np.cumsum(S, axis=1, dtype=U64, out=S)
    elif k == 2:    # d3 = (0, 1): down each column
        np.cumsum(S, axis=0, dtype=U64, out=S)
    elif k == 1:    # d2 = (1, 1): S(x, y) += S(x-1, y-1)
        for y in range(1, Hp):
            S[y, 1:] += S[y - 1, :-1]
    elif k == 3:    # d4 = (-1, 1): S(x, y) += S(x+1, y-1)
        for y in range(1, Hp):
            S[y, :-1] += S[y - 1, 1:]


def _scan128(S: U128, k: int) -> None:
    Hp, Wp = S.lo.shape
    if k == 0:
        for x in range(1, Wp):
            S[:, x] = S[:, x] + S[:, x - 1]
    elif k == 2:
        for y in range(1, Hp):
            S[y, :] = S[y, :] + S[y - 1, :]
    elif k == 1:
        for y in range(1, Hp):
            S[y, 1:] = S[y, 1:] + S[y - 1, :-1]
    elif k == 3:
        for y in range(1, Hp):
            S[y, :-1] = S[y, :-1] + S[y - 1, 1:]


SCAN_ORDER = (0, 2, 1, 3)  # d1, d3, d2, d4


def preintegrate(fq_ext: np.ndarray, n: int, bits: int = 64):
    """n-fold running sums along every direction, mod 2^bits.

    fq_ext: integer image on the padded domain (int64 or Python ints).
    Returns a uint64 array (bits=64), a uint32 array (bits=32) or a U128
    (bits=128).  Mod 2^32 the sums are the mod-2^64 sums reduced (reduction
    mod 2^32 is a ring homomorphism of Z/2^64), which is how bits=32 is
    computed.
    """
    if bits == 32:
        with np.errstate(over="ignore"):
            return (preintegrate(fq_ext, n, 64) & U64(0xFFFFFFFF)).astype(np.uint32)
    if bits == 64:
        if fq_ext.dtype == object:
            S = np.vectorize(lambda v: int(v) & MASK64, otypes=[object])(fq_ext).astype(U64)
        else:
            S = fq_ext.astype(np.int64).view(U64).copy()
        with np.errstate(over="ignore"):
            for k in SCAN_ORDER:
                for _ in range(n):
                    _scan64(S, k)
        return S
    if bits == 128:
        S = U128.from_ints(fq_ext.astype(object))
        for k in SCAN_ORDER:
            for _ in range(n):
                _scan128(S, k)
        return S
    raise ValueError(bits)


# ------------------------------ taps ---------------------------------------

def tap_weights(n: int):
    """[(t, w_t)] for t in {0..n}^4, w_t = prod_k (-1)^t_k C(n, t_k)."""
    out = []
    for t in itertools.product(range(n + 1), repeat=4):
        w = 1
        for tk in t:
            w *= (-1) ** tk * comb(n, tk)
        out.append((t, w))
    return out


def taps(S, Lfield: np.ndarray, n: int, R: int, H: int, W: int, bits: int = 64):
    """Signed exact accumulators acc[H][W] from the running sums S.

    Returns int64 (bits=64, and bits=32: the accumulator mod 2^32 read as a
    signed 32-bit value) or object (bits=128) arrays.
    """
    if bits == 32:   # the same combination mod 2^32
        with np.errstate(over="ignore"):
            acc = taps(np.asarray(S).astype(U64), Lfield, n, R, H, W, 64)
        return (acc.view(U64) & U64(0xFFFFFFFF)).astype(np.uint32).view(np.int32).astype(np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    L = Lfield.astype(np.int64)
    c = (n * (L - 1)) // 2
    base_x = xx + R + c[0] + c[1] - c[3]
    base_y = yy + R + c[1] + c[2] + c[3]
    if bits == 64:
        acc = np.zeros((H, W), dtype=U64)
    else:
        acc = _zeros_like_u128((H, W))
    with np.errstate(over="ignore"):
        for t, w in tap_weights(n):
            tx = base_x - t[0] * L[0] - t[1] * L[1] + t[3] * L[3]
            ty = base_y - t[1] * L[1] - t[2] * L[2] - t[3] * L[3]
            g = S[ty, tx]
            if bits == 64:
                if w >= 0:
                    acc += U64(w) * g
                else:
                    acc -= U64(-w) * g
            else:
                for _ in range(abs(w)):
                    acc = acc + g if w > 0 else acc - g
    if bits == 64:
        return acc.view(np.int64)
    return acc.to_signed_ints()


# --------------------------- whole filter ----------------------------------

def masses(Lfield: np.ndarray, n: int) -> np.ndarray:
    """D = prod_k L_k^n per pixel (int64 when it fits, else Python ints)."""
    H, W = Lfield.shape[1:]
    logmax = float((n * np.log2(np.maximum(Lfield, 1).astype(np.float64))).sum(axis=0).max(initial=0))
    if logmax < 62:
        D = np.ones((H, W), dtype=np.int64)
        for k in range(4):
            D *= Lfield[k].astype(np.int64) ** n
        return D
    D = np.empty((H, W), dtype=object)
    for y in range(H):
        for x in range(W):
            D[y, x] = kernel_mass(Lfield[:, y, x], n)
    return D


def filter_modular(f: np.ndarray, cov: np.ndarray, n: int, boundary: int, q: int,
                   bits: int = 64, out_dtype=np.float32, R: int | None = None,
                   rule: str = "corrected", return_all: bool = False):
    """Whole forward filter: steps, extension, quantisation, running sums, taps,
    final rounding.  cov is float32 [3][H][W] (C11, C12, C22)."""
    H, W = f.shape
    L, flags = params.integer_steps(cov[0], cov[1], cov[2], n, rule)
    if R is None:
        R = max(int(params.reach(L, n).max(initial=0)), 3 * n)
    else:
        # a pixel whose taps would leave the padded domain falls back to the
        # identity steps (the library reports it as out of reach)
        far = params.reach(L, n) > R
        L = np.where(far[None], 1, L)
    fq = quantize(f, q, as_object=(bits == 128))
    fe = extend_image(fq, R, boundary)
    S = preintegrate(fe, n, bits)
    acc = taps(S, L, n, R, H, W, bits)
    D = masses(L, n)
    out = finalize(acc, D, q, out_dtype)
    if return_all:
        return dict(out=out, L=L, flags=flags, R=R, S=S, acc=acc, D=D)
    return out
