"""CPU oracle for the space-variant box-spline filter -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct restatement of what the
filter computes, written from the paper (Chaudhury & Sanyal, "Improvements on
'Fast space-variant elliptical filtering using box splines'").  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  The CUDA library never links, imports or calls anything here,
and nothing here imports the CUDA library: the two share no code.

Modules
-------
params    covariance <-> scale-vector geometry, the minimum-kurtosis scale
          solve, step rounding, elongation bound e(phi).
kernels   discrete box-spline kernels and the direct (definition) filter.
modular   the paper's pipeline -- running sums, then finite differences --
          in exact two's-complement modular arithmetic.
gaussian  Gaussian-approximation errors of continuous box splines (Theorem 1,
          Table 2) by Parseval.
backward  the adjoint of the integer-step filter with respect to the image.
continuous  the continuous-step filter (interpolated taps, Section 2.3) and
          the derivative of its output with respect to the covariance field.
two_pass  Algorithm 1: an isotropic pass, then the space-variant residual pass.
sampled   the sampled continuous box spline: the filter of the paper's running
          sums interpolated by the grid box spline (eq. "interpolation").
config    the padding R, the automatic fraction bits q and element width:
          the configuration rules a run fixes before any arithmetic, so the
          tests check the library's choice instead of taking it.
knight    the second box spline beta'_a on the directions (2,1), (1,2), (-1,2),
          (-2,1) (Algorithm 3, Table 1) and the pair switched by sector
          (Algorithm 2).

Parity status of each function is stated in its docstring; "parity unpinned"
marks a function with no independent pin.
"""
from . import params, kernels, modular, gaussian, backward, continuous, two_pass, knight, sampled, config  # noqa: F401
