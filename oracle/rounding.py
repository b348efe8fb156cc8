"""Fixed-point quantisation of the input and the single final rounding.

Oracle module (test infrastructure only; see the package docstring).

The paper does not fix a number format.  The reading used here: the input is
quantised once, Q(f) = round-half-even(f 2^q), every later step is exact
integer arithmetic, and the only other rounding is the final division of the
exact accumulator acc by 2^q D, D = prod_k L_k^n the kernel mass:

    float32 output:  RN32( RN32(acc) * 2^-q ) / RN32(D)    (float32 divide)
    float64 output:  RN64( RN64(acc) * 2^-q ) / RN64(D)    (float64 divide)

RNxx(integer) is round-to-nearest-even of an exact integer; the scaling by
2^-q is exact.  The relative error against the exact rational acc/(2^q D) is
at most 3 units in the last place of the output format.
"""
from __future__ import annotations

import math

import numpy as np


def quantize(f: np.ndarray, q: int, as_object: bool = False) -> np.ndarray:
    """Q(f) = round-half-even(f * 2^q) exactly, as int64 (or Python ints).

    uint8 input: f << q.  float input: f is widened to float64 (exact), scaled
    by 2^q (exact barring overflow) and rounded half-to-even (numpy.rint).
    """
    if f.dtype == np.uint8:
        g = f.astype(object) * (1 << q) if as_object else f.astype(np.int64) << q
        return g
    x = f.astype(np.float64) * math.ldexp(1.0, q)
    x = np.rint(x)
    if as_object or np.abs(x).max(initial=0.0) >= 2.0 ** 62:
        return np.vectorize(lambda v: int(v), otypes=[object])(x)
    return x.astype(np.int64)


def rn_f32_int(a: int) -> np.float32:
    """Round an exact Python integer to the nearest float32, ties to even."""
    a = int(a)
    if a == 0:
        return np.float32(0.0)
    sgn = -1.0 if a < 0 else 1.0
    m = -a if a < 0 else a
    bl = m.bit_length()
    if bl <= 24:
        return np.float32(sgn * float(m))
    sh = bl - 24
    top = m >> sh
    rem = m - (top << sh)
    half = 1 << (sh - 1)
    if rem > half or (rem == half and (top & 1)):
        top += 1
    return np.float32(sgn * math.ldexp(float(top), sh))


def rn_f64_int(a: int) -> np.float64:
    """Round an exact Python integer to the nearest float64, ties to even.

    CPython's int -> float conversion is correctly rounded (half to even).
    """
    return np.float64(float(int(a)))


def _rn32_array(a: np.ndarray) -> np.ndarray:
    """Vectorised rn_f32_int for int64 arrays (exact, no double rounding)."""
    a = np.asarray(a, dtype=np.int64)
    neg = a < 0
    m = np.where(neg, -(a + 1), a).astype(np.uint64) + neg.astype(np.uint64)  # |a| without overflow
    # bit length of m
    e = np.frexp(m.astype(np.float64))[1].astype(np.int64)
    e = np.where(m == 0, 0, e)
    e = np.where((m > 0) & ((m >> np.maximum(e - 1, 0).astype(np.uint64)) == 0), e - 1, e)
    sh = np.maximum(e - 24, 0)
    shu = sh.astype(np.uint64)
    top = m >> shu
    rem = m - (top << shu)
    half = np.where(sh > 0, np.uint64(1) << np.maximum(sh - 1, 0).astype(np.uint64), np.uint64(0))
    up = (sh > 0) & ((rem > half) | ((rem == half) & ((top & np.uint64(1)) == 1)))
    top = top + up.astype(np.uint64)
    val = np.ldexp(top.astype(np.float64), sh)
    val = np.where(neg, -val, val)
    return val.astype(np.float32)


def finalize(acc, D, q: int, out_dtype) -> np.ndarray:
    """Apply the output rule to exact accumulators acc and masses D.

    acc, D: int64 arrays or object arrays of Python ints (same shape).
    """
    out_dtype = np.dtype(out_dtype)
    acc = np.asarray(acc)
    D = np.asarray(D)
    if out_dtype == np.float32:
        if acc.dtype == np.int64:
            x = _rn32_array(acc)
        else:
            x = np.vectorize(rn_f32_int, otypes=[np.float32])(acc)
        if D.dtype == np.int64 and (D < (1 << 24)).all():
            y = D.astype(np.float32)
        else:
            y = np.vectorize(rn_f32_int, otypes=[np.float32])(D.astype(object))
        scale = np.float32(math.ldexp(1.0, -q))
        return ((x * scale).astype(np.float32) / y).astype(np.float32)
    if out_dtype == np.float64:
        x = np.vectorize(rn_f64_int, otypes=[np.float64])(acc.astype(object))
        y = np.vectorize(rn_f64_int, otypes=[np.float64])(D.astype(object))
        return (x * math.ldexp(1.0, -q)) / y
    raise ValueError(out_dtype)
