"""Synthetic workloads for the space-variant box-spline filter.

Every generator is seeded and deterministic (``numpy.random.default_rng``), so
the CPU oracle and the GPU path receive identical bits.  The shapes and value
distributions follow the workloads the filter is benchmarked on:

* a uniform i.i.d. image in [0, 255] (float64),
* a "blob" image: a sum of isotropic Gaussian blobs (sigma 5-60 px,
  amplitude U[0,1], uniformly placed centres) plus N(0, 0.05^2) noise,
* the same blob image quantised to uint8 with a uniform dither,
* covariance fields given as three float32 planes (C11, C12, C22), built
  from a per-pixel size sigma, anisotropy ratio rho and major-axis angle
  theta (trace 2 sigma^2, eigenvalue ratio rho),
* smooth random fields (white noise low-passed with a Gaussian in the
  Fourier domain, then bilinearly upsampled and mapped to a range).

Covariance fields are laid out SoA, ``[3][H][W]`` float32 contiguous.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_image(H: int, W: int, seed: int = 0, lo: float = 0.0, hi: float = 255.0) -> np.ndarray:
    """i.i.d. uniform float64 image in [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(H, W)).astype(np.float64)


def random_integer_image(H: int, W: int, seed: int = 0, lo: int = -1000, hi: int = 1000) -> np.ndarray:
    """i.i.d. integer-valued float64 image (exactly representable in fp32 too)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi, size=(H, W)).astype(np.float64)


def blob_image(H: int, W: int, seed: int = 0, n_blobs: int = 200,
               sigma_range=(5.0, 60.0), noise_sd: float = 0.05,
               dtype=np.float32) -> np.ndarray:
    """Sum of ``n_blobs`` isotropic Gaussian blobs plus white Gaussian noise.

    Each blob has sigma ~ U[sigma_range], amplitude ~ U[0,1] and a centre
    uniform over the image.  Blobs are evaluated separably inside a +-5 sigma
    window, which changes the sum by less than exp(-12.5) of a blob's peak.
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), dtype=np.float64)
    sig = rng.uniform(sigma_range[0], sigma_range[1], size=n_blobs)
    amp = rng.uniform(0.0, 1.0, size=n_blobs)
    cx = rng.uniform(0.0, W, size=n_blobs)
    cy = rng.uniform(0.0, H, size=n_blobs)
    for s, a, x0, y0 in zip(sig, amp, cx, cy):
        r = int(math.ceil(5.0 * s))
        xa, xb = max(0, int(x0) - r), min(W, int(x0) + r + 1)
        ya, yb = max(0, int(y0) - r), min(H, int(y0) + r + 1)
        if xa >= xb or ya >= yb:
            continue
        gx = np.exp(-0.5 * ((np.arange(xa, xb) - x0) / s) ** 2)
        gy = np.exp(-0.5 * ((np.arange(ya, yb) - y0) / s) ** 2)
        img[ya:yb, xa:xb] += a * np.outer(gy, gx)
    img += rng.normal(0.0, noise_sd, size=(H, W))
    return img.astype(dtype)


def blob_image_u8(H: int, W: int, seed: int = 0, n_blobs: int = 200) -> np.ndarray:
    """The blob image scaled to [0, 255], dithered with U(-1/2, 1/2), rounded, clipped."""
    f = blob_image(H, W, seed=seed, n_blobs=n_blobs, dtype=np.float64)
    lo, hi = float(f.min()), float(f.max())
    g = (f - lo) * (255.0 / max(hi - lo, 1e-30))
    rng = np.random.default_rng(seed + 7919)
    g = g + rng.uniform(-0.5, 0.5, size=g.shape)
    return np.clip(np.rint(g), 0, 255).astype(np.uint8)


def covariance_from_axes(sigma, rho, theta) -> np.ndarray:
    """Covariance planes with trace 2 sigma^2, eigenvalue ratio rho, major axis at theta.

    Builds C = k R(theta) diag(rho, 1) R(theta)^T with k = 2 sigma^2 / (1 + rho),
    so an isotropic field (rho = 1) gives C = sigma^2 I.  Returns float32
    ``[3][...]`` planes (C11, C12, C22); the arithmetic is done in float64.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    sigma, rho, theta = np.broadcast_arrays(sigma, rho, theta)
    k = 2.0 * sigma * sigma / (1.0 + rho)
    c, s = np.cos(theta), np.sin(theta)
    c11 = k * (rho * c * c + s * s)
    c22 = k * (rho * s * s + c * c)
    c12 = k * (rho - 1.0) * s * c
    return np.ascontiguousarray(np.stack([c11, c12, c22]), dtype=np.float32)


def constant_cov_field(H: int, W: int, c11: float, c12: float, c22: float) -> np.ndarray:
    """Space-invariant covariance field as ``[3][H][W]`` float32."""
    out = np.empty((3, H, W), dtype=np.float32)
    out[0], out[1], out[2] = c11, c12, c22
    return out


def diagonal_ramp_cov_field(H: int, W: int, sigma_lo: float = 1.0, sigma_hi: float = 16.0,
                            rho_lo: float = 1.0, rho_hi: float = 4.0) -> np.ndarray:
    """Space-variant field: sigma rises linearly across x, theta oscillates in y,
    the anisotropy ratio rises along the main diagonal.

    sigma(x) = sigma_lo + (sigma_hi - sigma_lo) x / (W - 1)
    theta(x, y) = pi (0.5 + 0.5 sin(2 pi y / H))
    rho(x, y) = rho_lo + (rho_hi - rho_lo) (x + y) / (W + H - 2)
    """
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    sigma = sigma_lo + (sigma_hi - sigma_lo) * x / max(W - 1, 1)
    theta = math.pi * (0.5 + 0.5 * np.sin(2.0 * math.pi * y / H))
    rho = rho_lo + (rho_hi - rho_lo) * (x + y) / max(W + H - 2, 1)
    return covariance_from_axes(sigma, rho, theta)


def _bilinear_upsample(g: np.ndarray, H: int, W: int) -> np.ndarray:
    """Bilinear interpolation of g onto an H x W grid spanning the same extent."""
    h, w = g.shape
    ys = np.linspace(0.0, h - 1.0, H)
    xs = np.linspace(0.0, w - 1.0, W)
    y0 = np.minimum(np.floor(ys).astype(np.int64), h - 2) if h > 1 else np.zeros(H, np.int64)
    x0 = np.minimum(np.floor(xs).astype(np.int64), w - 2) if w > 1 else np.zeros(W, np.int64)
    wy = (ys - y0)[:, None]
    wx = (xs - x0)[None, :]
    y1 = np.minimum(y0 + 1, h - 1)
    x1 = np.minimum(x0 + 1, w - 1)
    top = g[y0][:, x0] * (1 - wx) + g[y0][:, x1] * wx
    bot = g[y1][:, x0] * (1 - wx) + g[y1][:, x1] * wx
    return np.ascontiguousarray(top * (1 - wy) + bot * wy)


def smooth_field(H: int, W: int, seed: int, lo: float, hi: float,
                 corr_frac: float = 1.0 / 8.0, coarse: int = 16) -> np.ndarray:
    """Smooth random field mapped affinely onto [lo, hi] (float64).

    White noise on a grid ``coarse`` times smaller than the image is low-passed
    by a Gaussian of correlation length ``corr_frac`` x side in the Fourier
    domain, normalised to [0, 1], bilinearly upsampled to (H, W) and mapped.
    """
    rng = np.random.default_rng(seed)
    h = max(4, -(-H // coarse))
    w = max(4, -(-W // coarse))
    noise = rng.standard_normal((h, w))
    ky = np.fft.fftfreq(h)[:, None]
    kx = np.fft.fftfreq(w)[None, :]
    ell = corr_frac * max(h, w)
    filt = np.exp(-2.0 * (math.pi * ell) ** 2 * (kx * kx + ky * ky))
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
    g = (g - g.min()) / max(g.max() - g.min(), 1e-30)
    up = _bilinear_upsample(g, H, W)
    return lo + (hi - lo) * up


def random_cov_field(H: int, W: int, seed: int, sigma_range, rho_range) -> np.ndarray:
    """Smooth random covariance field: smooth sigma and rho fields in the given
    ranges and a smooth orientation field covering [0, pi)."""
    sigma = smooth_field(H, W, seed, sigma_range[0], sigma_range[1])
    rho = smooth_field(H, W, seed + 1, rho_range[0], rho_range[1])
    theta = smooth_field(H, W, seed + 2, 0.0, math.pi)
    return covariance_from_axes(sigma, rho, theta)


def param_fields_logsig_theta_logrho(H: int, W: int, seed: int,
                                     logsig_range=(0.0, 3.0), logrho_range=(0.0, 1.1)) -> np.ndarray:
    """Three smooth float32 parameter planes (log sigma, theta, log rho)."""
    a = smooth_field(H, W, seed, logsig_range[0], logsig_range[1])
    b = smooth_field(H, W, seed + 1, 0.0, math.pi)
    c = smooth_field(H, W, seed + 2, logrho_range[0], logrho_range[1])
    return np.ascontiguousarray(np.stack([a, b, c]), dtype=np.float32)


def batch_sizes_loguniform(B: int, seed: int = 1, lo: int = 128, hi: int = 2048):
    """B (H, W) pairs with H and W drawn independently log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    hs = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))).astype(int)
    ws = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))).astype(int)
    return [(int(h), int(w)) for h, w in zip(hs, ws)]
