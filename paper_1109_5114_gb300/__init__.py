"""GB300-native O(1) space-variant box-spline filtering.

The compute path is libbsf.so (CUDA for sm_103a) behind the C ABI of
include/bsf.h; ``paper_1109_5114_gb300.bsf`` is its ctypes binding.  Build the
library with ``paper_1109_5114_gb300.build.build()``.
"""

__all__ = ["build", "bsf"]
