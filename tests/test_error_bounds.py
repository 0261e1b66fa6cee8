"""Host checks of the rounding bounds the tensor-core kernels rely on.

The tensor-core assignment forms x.c from FP16 parts: every row of X is
scaled by a power of two that puts its largest coordinate in [2^14, 2^15),
all of C by one such power of two, and each scaled value v splits into
hi = fp16(v) and lo = fp16(v - hi); x.c ~ x_hi.c_hi + x_hi.c_lo + x_lo.c_hi.
Its margin assumes that this product is within (3 + 3 * 2^-11) * 2^-22 of
sum |x_t c_t| plus 2^-27 of ||x||^2 + ||c||^2.  Here numpy's float16 plays
the tensor core's operands (products and sums in FP64, so only the split's
own error is measured).

The tensor-core leaf scan's filter reads each row as TF32 and splits each
query into an exact TF32 part and a remainder read as TF32; its margin
assumes the product within (2^-10 + 2^-20 + 2^-30) of sum |x_t q_t|, for
either reading of FP32 as TF32 (truncation or rounding to nearest).
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


def _tf32(v, mode):
    """FP32 -> TF32 (10 explicit mantissa bits) by truncation or round to
    nearest; the tensor core's reading is one of the two."""
    b = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32)
    if mode == "rn":
        b = b + np.uint32(0x1000)
    return (b & np.uint32(0xFFFFE000)).view(np.float32)


@pytest.mark.parametrize("mode", ["trunc", "rn"])
@pytest.mark.parametrize("seed", range(3))
def test_tf32_leaf_scan_product_stays_within_its_bound(seed, mode):
    # The leaf scan's tensor-core product reads each row as TF32 and each
    # query as q_hi (low 13 mantissa bits cleared) plus q_lo = q - q_hi read
    # as TF32: x.q ~ x~.q_hi + x~.q_lo~.  Its filter margin assumes this is
    # within (2^-10 + 2^-20 + 2^-30) of sum |x_t q_t| before the FP32
    # accumulation terms (products and sums in FP64 here).
    rng = np.random.default_rng(100 + seed)
    worst = 0.0
    for _ in range(200):
        d = int(rng.choice([32, 64]))
        q = (rng.normal(size=d) * rng.uniform(1e-2, 1e2)).astype(np.float32)
        X = (rng.normal(size=(64, d)) * rng.uniform(1e-2, 1e2)
             + rng.uniform(-10, 10, size=d)).astype(np.float32)
        qhi = (q.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
        qlo = (q - qhi).astype(np.float32)
        assert np.array_equal(qhi.astype(np.float64) + qlo, q.astype(np.float64))  # exact split
        xt = _tf32(X, mode).astype(np.float64)
        approx = xt @ qhi.astype(np.float64) + xt @ _tf32(qlo, mode).astype(np.float64)
        exact = X.astype(np.float64) @ q.astype(np.float64)
        bound = (2.0 ** -10 + 2.0 ** -20 + 2.0 ** -30) * np.abs(X.astype(np.float64) * q).sum(1)
        worst = max(worst, float((np.abs(approx - exact) / bound).max()))
    assert 0.1 < worst <= 1.0, worst   # the bound holds and is not vacuous
