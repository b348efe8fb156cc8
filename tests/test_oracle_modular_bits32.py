"""Pins of the 32-bit modular mode of the oracle (modular.preintegrate /
taps with bits=32, and the same for the second direction set): equal to the
direct correlation while the accumulator fits a signed 32-bit value, and
wrapped (hence different) beyond."""
import numpy as np
import pytest

from oracle import kernels, knight as kn, modular
from oracle.rounding import quantize
from workloads import synth


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("boundary", [0, 2])
def test_bits32_equals_direct_within_the_bound(n, boundary):
    H, W = 15, 18
    f = synth.random_integer_image(H, W, seed=n, lo=0, hi=255).astype(np.float32)
    cov = synth.random_cov_field(H, W, seed=n + 1, sigma_range=(0.5, 1.5), rho_range=(1.0, 2.0))
    r = modular.filter_modular(f, cov, n, boundary, q=0, bits=32, out_dtype=np.float64, return_all=True)
    assert int(np.abs(r["acc"]).max()) < 2 ** 31
    ref = kernels.correlate_exact(quantize(f, 0), r["L"], n, boundary)
    assert (r["acc"].astype(object) == ref).all()
    r2 = kn.filter_modular_k(f, cov, n, boundary, q=0, bits=32, out_dtype=np.float64, return_all=True)
    ref2 = kn.correlate_exact_k(quantize(f, 0), r2["L"], n, boundary)
    assert (r2["acc"].astype(object) == ref2).all()


def test_bits32_wraps_beyond_the_bound():
    H, W = 12, 12
    f = np.full((H, W), 255.0, np.float32)
    cov = synth.constant_cov_field(H, W, 9.0, 0.0, 9.0)
    a32 = modular.filter_modular(f, cov, 3, 2, q=10, bits=32, return_all=True)["acc"]
    a64 = modular.filter_modular(f, cov, 3, 2, q=10, bits=64, return_all=True)["acc"]
    assert int(np.abs(a64).max()) >= 2 ** 31
    assert (a32 != a64).any()
    assert ((a64 - a32) % (1 << 32) == 0).all()
