"""Host checks of the rounding bounds the tensor-core kernels rely on.

The tensor-core assignment forms x.c from FP16 parts: every row of X is
scaled by a power of two that puts its largest coordinate in [2^14, 2^15),
all of C by one such power of two, and each scaled value v splits into
hi = fp16(v) and lo = fp16(v - hi); x.c ~ x_hi.c_hi + x_hi.c_lo + x_lo.c_hi.
Its margin assumes that this product is within (3 + 3 * 2^-11) * 2^-22 of
sum |x_t c_t| plus 2^-27 of ||x||^2 + ||c||^2.  Here numpy's float16 plays
the tensor core's operands (products and sums in FP64, so only the split's
own error is measured).
"""

import numpy as np
import pytest


def _split(v, m):
    e = 14 - int(np.floor(np.log2(m))) if m > 0 else 0
    w = (v * np.float32(2.0 ** e)).astype(np.float32)
    hi = w.astype(np.float16)
    lo = (w - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float64), lo.astype(np.float64), 2.0 ** -e


@pytest.mark.parametrize("seed", range(4))
def test_fp16_three_product_split_stays_within_its_bound(seed):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(100):
        d = int(rng.integers(1, 65))
        x = (rng.normal(size=d) * rng.uniform(1e-3, 1e3)).astype(np.float32)
        x[rng.random(d) < 0.2] *= np.float32(1e-5)   # small coordinates: subnormal lo parts
        c = (rng.normal(size=(40, d)) * rng.uniform(1e-3, 1e3)).astype(np.float32)
        hx, lx, ix = _split(x, np.abs(x).max())
        hc, lc, ic = _split(c, np.abs(c).max())           # one scale for all of C
        approx = (hx * hc + hx * lc + lx * hc).sum(1) * ix * ic
        x64, c64 = x.astype(np.float64), c.astype(np.float64)
        exact = c64 @ x64
        bound = ((3 + 3 * 2.0 ** -11) * 2.0 ** -22 * np.abs(c64 * x64).sum(1)
                 + 2.0 ** -27 * ((x64 ** 2).sum() + (c64 ** 2).sum(1)))
        worst = max(worst, float((np.abs(approx - exact) / bound).max()))
    assert worst <= 1.0, worst
