"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package builds images and covariance fields only.  It holds none of the
filter's arithmetic (no running sums, no finite differences, no scale solve),
so the CUDA path and the CPU oracle can both consume its outputs without
sharing any step of the method.
"""
from .synth import (  # noqa: F401
    uniform_image,
    blob_image,
    blob_image_u8,
    covariance_from_axes,
    constant_cov_field,
    diagonal_ramp_cov_field,
    smooth_field,
    random_cov_field,
    param_fields_logsig_theta_logrho,
    random_integer_image,
    batch_sizes_loguniform,
)
