"""Gaussian approximation by continuous box splines (Theorem 1, Table 2).

Oracle module (test infrastructure only; see the package docstring).

A box distribution of width a along the unit vector u has Fourier transform
sinc(a (w . u) / 2), sinc(t) = sin(t)/t, so the box spline with scales a_k
along directions u_k has transform prod_k sinc(a_k (w . u_k)/2) (Section 1.1,
eq. "boxSpline").  The Gaussian of covariance C has transform
exp(-w^T C w / 2).  By Parseval the normalised L2 error used in Section 3,
||beta - g||_2 / ||g||_2, is computed in the Fourier domain:

    err^2 = int |beta^(w) - g^(w)|^2 dw / int |g^(w)|^2 dw,
    int |g^|^2 dw = pi / sqrt(det C).

The integral is a midpoint rule on a square grid (the integrand is even, so
only half the plane is summed), fine enough that the printed one-decimal
percentages are reproduced.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_directions(N: int):
    """theta_k = (k-1) pi / N, k = 1..N (Theorem 1)."""
    return [(math.cos(k * math.pi / N), math.sin(k * math.pi / N)) for k in range(N)]


CARTESIAN = uniform_directions(4)


def box_spline_ft(wx, wy, scales, dirs):
    """prod_k sinc(a_k (w . u_k) / 2) on arrays of frequencies."""
    out = np.ones_like(wx)
    for a, (ux, uy) in zip(scales, dirs):
        t = 0.5 * a * (wx * ux + wy * uy)
        out = out * np.sinc(t / math.pi)  # numpy sinc(x) = sin(pi x)/(pi x)
    return out


def normalized_l2_error(stages, C, wmax: float = 40.0, dw: float = 0.02) -> float:
    """||beta - g||_2 / ||g||_2 for beta = convolution of the given stages.

    stages: list of (scales, dirs); the box spline transforms multiply.
    C: 2x2 target covariance.  Frequencies are scaled by the target's size so
    the grid resolves it independently of units.
    """
    C = np.asarray(C, dtype=np.float64)
    s = math.sqrt(np.trace(C) / 2.0)
    # integrate in normalised frequency v = w * s
    n = int(round(wmax / dw))
    v1 = (np.arange(-n, n) + 0.5) * dw
    v2 = (np.arange(0, n) + 0.5) * dw          # half plane (even integrand)
    num = 0.0
    den = 0.0
    for i0 in range(0, len(v2), 256):
        vy = v2[i0:i0 + 256][:, None]
        vx = v1[None, :]
        wx, wy = vx / s, vy / s
        b = np.ones(np.broadcast(wx, wy).shape)
        for scales, dirs in stages:
            b = b * box_spline_ft(wx, wy, scales, dirs)
        g = np.exp(-0.5 * (C[0, 0] * wx * wx + 2 * C[0, 1] * wx * wy + C[1, 1] * wy * wy))
        num += float(((b - g) ** 2).sum())
        den += float((g * g).sum())
    return math.sqrt(num / den)


def isotropic_scales(sigma: float, N: int = 4):
    """a_k = sigma sqrt(24/N) for all k (Theorem 1 / eq. "boxSpline"); for N = 4
    this is sqrt(6) sigma (Section 1.1)."""
    return [sigma * math.sqrt(24.0 / N)] * N


def boxfilter_isotropic_error(sigma: float = 1.0, N: int = 4) -> float:
    """Error of the single isotropic box spline against the Gaussian sigma^2 I."""
    return normalized_l2_error([(isotropic_scales(sigma, N), uniform_directions(N))],
                               sigma * sigma * np.eye(2))


def algorithm1_isotropic_error(sigma: float = 1.0, frac: float = 0.5) -> float:
    """Error of Algorithm 1 for an isotropic target sigma^2 I.

    The pre-blur takes sigma0^2 = frac x (condition-2 bound); for an isotropic
    C the bound is sigma^2, and the residual sigma^2 - sigma0^2 is again
    isotropic, so both stages are isotropic box splines (scales sqrt(6) x
    their standard deviations).
    """
    s0 = math.sqrt(frac) * sigma
    s1 = math.sqrt(sigma * sigma - s0 * s0)
    return normalized_l2_error([(isotropic_scales(s0), CARTESIAN),
                                (isotropic_scales(s1), CARTESIAN)],
                               sigma * sigma * np.eye(2))


def box_spline_spatial(scales, dirs, half_width: float, h: float, pad: int = 4):
    """Samples of the continuous box spline on [-hw, hw]^2 with spacing h,
    by inverse FFT of its transform (zero-padded x pad to limit aliasing)."""
    m = int(round(2 * half_width / h))
    M = m * pad
    w = 2 * math.pi * np.fft.fftfreq(M, d=h)
    wx, wy = np.meshgrid(w, w)
    F = box_spline_ft(wx, wy, scales, dirs)
    img = np.real(np.fft.fftshift(np.fft.ifft2(F))) / (h * h)
    c = M // 2
    return img[c - m // 2:c + m // 2 + 1, c - m // 2:c + m // 2 + 1]


def gaussian_spatial(C, half_width: float, h: float):
    m = int(round(2 * half_width / h))
    x = (np.arange(m + 1) - m // 2) * h
    X, Y = np.meshgrid(x, x)
    Ci = np.linalg.inv(C)
    q = Ci[0, 0] * X * X + 2 * Ci[0, 1] * X * Y + Ci[1, 1] * Y * Y
    return np.exp(-0.5 * q) / (2 * math.pi * math.sqrt(np.linalg.det(C)))
