"""Configuration a filter run fixes before any arithmetic: the padding R and,
when the caller leaves them open, the fraction bits q and the element width.

Oracle module (test infrastructure only; see the package docstring).

These are the documented rules of the number format (the paper fixes none;
readings "number format" and "32-bit elements and the automatic width"),
computed here from the oracle's own step solve, so that a test can check the
library's choice against them instead of taking it from the library:

* R: the largest tap reach of the field's steps, at least 3n (and at least
  the reach of identity steps for the continuous and sampled steps).
* mass bound: the largest kernel mass of the field, as the float32 product
  the plan reduces (prod L^n for integer steps, prod M_k for the continuous
  steps with their 2^10-scaled weights).
* automatic q: the largest q with (vmax 2^q + 1/2) mass < 2^(b-2), written
  floor((b - 2) - log2 vmax - log2 mass) - 1 (two fewer bits for the
  continuous steps, whose derivative sums reach 3 vmax mass), capped at
  b - 28 (30 for 32-bit elements) and floored at 0.
* automatic width (BSF_FIX): the narrowest of 32, 64 and 128 bits (64 and
  128 for continuous or sampled steps) whose automatic q reaches
  q_t = 25 - ceil(log2 vmax) (0 for 8-bit images), or, with a fixed q, whose
  bound log2((vmax 2^q + 1/2) mass) < b - 2 holds.
"""
from __future__ import annotations

import math

import numpy as np

from . import params

_F = np.float32


def integer_masses_f32(L: np.ndarray, n: int) -> np.ndarray:
    """prod_k L_k^n per pixel as float32: m1 = f32(L1 L2) * f32(L3 L4), then
    m1 multiplied in n - 1 more times (float32 products)."""
    L = np.asarray(L, dtype=np.int64)
    m1 = (L[0] * L[1]).astype(_F) * (L[2] * L[3]).astype(_F)
    m = m1.astype(_F)
    for _ in range(1, n):
        m = (m * m1).astype(_F)
    return m


def continuous_masses_f32(Hs: np.ndarray, n: int) -> np.ndarray:
    """prod_k M_k per pixel as float32 (1 * M_1 * M_2 * M_3 * M_4), with M_k
    the exact mass of the continuous-step line kernel of H_k."""
    from .continuous import line_data
    Hs = np.asarray(Hs, dtype=np.int64)
    m = np.ones(Hs.shape[1:], dtype=_F)
    for k in range(4):
        u, inv = np.unique(Hs[k], return_inverse=True)
        Mk = np.array([line_data(int(h), n)[3] for h in u], dtype=object)
        m = (m * np.array([_F(int(v)) for v in Mk], dtype=_F)[inv.reshape(Hs.shape[1:])]).astype(_F)
    return m


def continuous_reach(Hs: np.ndarray, n: int) -> np.ndarray:
    """continuous.reach_d2 for a whole field (per distinct step, then mapped)."""
    from .continuous import line_taps
    Hs = np.asarray(Hs, dtype=np.int64)
    lo, hi = [], []
    for k in range(4):
        u, inv = np.unique(Hs[k], return_inverse=True)
        taps = [line_taps(int(h), n)[0] for h in u]
        lo.append(np.array([min(t) for t in taps], dtype=np.int64)[inv.reshape(Hs.shape[1:])])
        hi.append(np.array([max(t) for t in taps], dtype=np.int64)[inv.reshape(Hs.shape[1:])])
    x_min = lo[0] + lo[1] - hi[3]
    x_max = hi[0] + hi[1] - lo[3]
    y_min = lo[1] + lo[2] + lo[3]
    y_max = hi[1] + hi[2] + hi[3]
    return np.maximum(np.maximum(-x_min, x_max), np.maximum(-y_min, y_max))


def steps_and_reach(cov: np.ndarray, n: int, rule: str = "corrected", dirs: str = "cartesian",
                    kind: int = 0):
    """(per-pixel reach, float32 masses) of a float32 [3][H][W] field.

    rule: "corrected" | "paper" (integer steps), "d2" (continuous steps),
    "sampled" (order 1).  dirs: "cartesian" | "second" | "pair".  kind: 0 for
    (C11, C12, C22) planes, 1 for (log sigma, theta, log rho) planes."""
    from . import continuous, knight, sampled
    C11, C12, C22 = continuous.covariance_planes(cov, kind)
    if rule == "d2":
        Hs, _, _ = continuous.half_steps(C11, C12, C22, n)
        return continuous_reach(Hs, n), continuous_masses_f32(Hs, n)
    if rule == "sampled":
        Lq, _ = sampled.lambdas_q(C11, C12, C22)
        r0 = sampled.reach(Lq)
        m0 = (Lq[0].astype(_F) * Lq[1].astype(_F) * Lq[2].astype(_F) * Lq[3].astype(_F) * _F(2.0 ** -13)).astype(_F)
        if dirs == "cartesian":
            return r0, m0
        Lk, _ = sampled.lambdas_q_k(C11, C12, C22)
        r1 = sampled.reach_k(Lk)
        m1 = (Lk[0].astype(_F) * Lk[1].astype(_F) * Lk[2].astype(_F) * Lk[3].astype(_F)
              * _F(15.0 * 2.0 ** -5)).astype(_F)
        if dirs == "second":
            return r1, m1
        mask = knight.use_knight(C11, C12, C22)
        return np.where(mask, r1, r0), np.where(mask, m1, m0)
    L0, _ = params.integer_steps(C11, C12, C22, n, rule)
    if dirs == "cartesian":
        return params.reach(L0, n), integer_masses_f32(L0, n)
    L1, _ = knight.integer_steps_k(C11, C12, C22, n, rule)
    if dirs == "second":
        return knight.reach_k(L1, n), integer_masses_f32(L1, n)
    mask = knight.use_knight(C11, C12, C22)
    return (np.where(mask, knight.reach_k(L1, n), params.reach(L0, n)),
            np.where(mask, integer_masses_f32(L1, n), integer_masses_f32(L0, n)))


# the reach of identity steps for the continuous steps (samples at -3..1 for
# n = 2, -2..1 for n = 1 along every direction) and for the sampled box
# splines (lambda = 1 in every direction)
def _min_reach(rule: str, n: int, dirs: str) -> int:
    if rule == "d2":
        return 9 if n == 2 else 6
    if rule == "sampled":
        return 4 if dirs == "cartesian" else 10
    return 0


def padding(cov: np.ndarray, n: int, rule: str = "corrected", dirs: str = "cartesian", kind: int = 0) -> int:
    """R of a field: the largest reach, at least 3n and the identity steps' reach."""
    reach, _ = steps_and_reach(cov, n, rule, dirs, kind)
    return max(int(np.max(reach, initial=0)), 3 * n, _min_reach(rule, n, dirs))


def mass_bound(cov: np.ndarray, n: int, rule: str = "corrected", dirs: str = "cartesian", kind: int = 0) -> float:
    """Largest float32 kernel mass of the field (at least 1)."""
    _, m = steps_and_reach(cov, n, rule, dirs, kind)
    return max(float(np.max(m, initial=1.0)), 1.0)


def value_bound(img: np.ndarray) -> float:
    """max |f| as the library reduces it: 255 for 8-bit images, else the
    largest magnitude (float32 images widened exactly to float64)."""
    if img.dtype == np.uint8:
        return 255.0
    return float(np.abs(img.astype(np.float64)).max(initial=0.0))


def auto_frac_bits(vmax: float, mass: float, bits: int, continuous: bool = False) -> int:
    """The automatic q for elements of `bits` bits (before the floor at 0)."""
    lv = math.log2(vmax if vmax > 1e-300 else 1e-300)
    lm = math.log2(mass if mass > 1.0 else 1.0)
    q = math.floor((bits - 2) - lv - lm) - 1
    if continuous:
        q -= 2
    return min(q, 30 if bits == 32 else bits - 28)


def resolve(img: np.ndarray, mass: float, frac_bits: int = -1, bits: int | None = 64,
            continuous: bool = False, vmax: float | None = None, wide_only: bool | None = None):
    """(bits, q) a run takes: bits None means the automatic width (BSF_FIX);
    frac_bits < 0 means the automatic q.  vmax defaults to value_bound(img)
    (a caller's explicit value bound replaces it).  continuous: the
    continuous steps' two guard bits; wide_only (default: continuous): the
    automatic width starts at 64 bits (continuous and sampled steps)."""
    if wide_only is None:
        wide_only = continuous
    if vmax is None:
        vmax = value_bound(img)
    mass = max(mass, 1.0)
    if bits is None:
        qt = 0 if img.dtype == np.uint8 else 25 - math.ceil(math.log2(vmax if vmax > 1e-300 else 1e-300))
        bits = 128
        for b in ((64, 128) if wide_only else (32, 64, 128)):
            if frac_bits >= 0:
                fits = math.log2((vmax * math.ldexp(1.0, frac_bits) + 0.5) * mass) < b - 2
            else:
                fits = auto_frac_bits(vmax, mass, b, continuous) >= max(qt, 0)
            if fits:
                bits = b
                break
        if frac_bits >= 0:
            return bits, frac_bits
    if frac_bits >= 0:
        return bits, frac_bits
    return bits, max(auto_frac_bits(vmax, mass, bits, continuous), 0)
