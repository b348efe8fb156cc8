"""The library's usage example (one image filtered on its own and by
Algorithm 1's two passes) runs as written, and both of its calls agree bit
for bit with the oracle on sampled rows (each checked on a band of rows that
reaches two paddings beyond them, so the band's own edges are out of reach
of both passes).  R and q come from the oracle's rules, checked against the
library's."""
import numpy as np
import pytest

from oracle import config, modular, two_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_5114_gb300 import build
    build.build()


def test_usage_example():
    import torch
    from paper_1109_5114_gb300 import bsf

    torch.manual_seed(0)
    # --- the usage example ---
    H, W = 2048, 2048
    img = torch.rand(H, W, device="cuda")
    cov = torch.empty(3, H, W, device="cuda")
    cov[0] = 9.0; cov[1] = 2.0; cov[2] = 4.0  # noqa: E702
    f = bsf.BoxSplineFilter(H, W, 2, "symmetric", value_bound=1.0)
    out = f.filter(img, cov)
    torch.cuda.synchronize()
    info1 = f.info()
    out2 = f.filter_two_pass(img, cov, 0.5)
    torch.cuda.synchronize()
    assert f.status() == 0
    info2 = f.info()
    f.close()
    # --- against the oracle ---
    im = img.cpu().numpy()
    cv = cov.cpu().numpy()
    o1, o2 = out.cpu().numpy(), out2.cpu().numpy()
    # the plan of the first call (its R and mass bound) serves the second;
    # the value bound 1.0 fixes q
    R = config.padding(cv, 2)
    q = max(config.auto_frac_bits(1.0, config.mass_bound(cv, 2), 64), 0)
    assert (info1.R, info1.frac_bits) == (R, q) == (info2.R, info2.frac_bits)
    for y0 in (0, 1500, H - 8):
        lo, hi = max(0, y0 - 2 * R), min(H, y0 + 8 + 2 * R)
        band = modular.filter_modular(im[lo:hi], cv[:, lo:hi], 2, 2, q=q, bits=64,
                                      out_dtype=np.float32, R=R)
        np.testing.assert_array_equal(o1[y0:y0 + 8], band[y0 - lo:y0 - lo + 8])
        band2, _, _ = two_pass.algorithm1(im[lo:hi], cv[:, lo:hi], 2, 2, q=q, R=R)
        np.testing.assert_array_equal(o2[y0:y0 + 8], band2[y0 - lo:y0 - lo + 8])
