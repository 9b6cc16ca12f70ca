"""The two numerical facts the FP16 hi/lo Legendre table kernels rest on, checked
on the CPU:

* the table scale 2^9: every orthonormal associated Legendre value obeys
  |lambda_lm(theta)| <= sqrt((2l+1)/(4 pi)) (the addition theorem,
  sum_m |Y_lm|^2 = (2l+1)/(4 pi)), so 2^9 |lambda| < 2^14 below l = 4096, inside
  the FP16 range with room for the rounding of hi; checked on the oracle's own
  values on MW rings;
* the split with a power-of-two column scale: x s = hi + lo with hi = fp16(x s),
  lo = fp16(x s - hi) (round to nearest), s = 2^(12 - e) for the column maximum in
  [2^e, 2^(e+1)), carries every value to 2^-22 of itself or, for values far below
  the column maximum, to 2^-37 of that maximum; a model in numpy float16 on columns
  that span 1e-30 .. 1e30 and 40 binary orders within a column.
"""
import math

import numpy as np

from oracle import sht


def test_legendre_values_obey_the_addition_theorem_bound():
    N = 256
    ts = [0, 1, N // 7, N // 3, N // 2, N - 2, N - 1]
    worst = 0.0
    for m in range(0, N, 5):
        l = np.arange(m, N)
        bound = np.sqrt((2 * l + 1) / (4 * math.pi))
        for t in ts:
            lam = sht.legendre_at(m, N, t)
            worst = max(worst, float(np.max(np.abs(lam) / bound)))
    assert 0.1 < worst <= 1.0 + 1e-12
    # the scale used by the tables keeps |hi| below 2^14 for every l < 4096
    assert 512.0 * math.sqrt((2 * 4095 + 1) / (4 * math.pi)) < 2.0 ** 14


def _colscale(mx):
    """The kernels' column scale: 2^(12 - floor(log2 mx)), 1 for a zero column."""
    if not mx > 0:
        return 1.0
    e = math.floor(math.log2(mx))
    return 2.0 ** min(126, max(-126, 12 - e))


def _split(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float64)).astype(np.float16)
    return hi, lo


def test_fp16_split_with_column_scales_keeps_22_bits():
    rng = np.random.Generator(np.random.PCG64(11))
    for mag in (1e-30, 1.0, 1e30):
        # one column: values spread over 40 binary orders below its maximum
        col = mag * rng.standard_normal(4096) * 2.0 ** rng.uniform(-40, 0, 4096)
        col = col.astype(np.float32).astype(np.float64)
        mx = float(np.max(np.abs(col)))
        s = _colscale(mx)
        xs = col * s
        assert np.max(np.abs(xs)) < 2.0 ** 13
        hi, lo = _split(xs)
        assert np.all(np.isfinite(hi.astype(np.float64)))
        rec = (hi.astype(np.float64) + lo.astype(np.float64)) / s
        err = np.abs(rec - col)
        bound = np.maximum(2.0 ** -22 * np.abs(col), 2.0 ** -37 * mx)
        assert np.all(err <= bound), float(np.max(err / bound))
        # values within 2^-3 of the maximum keep the full 22 bits
        big = np.abs(col) >= mx / 8
        assert np.all(err[big] <= 2.0 ** -22 * np.abs(col[big]))


def test_split_product_against_fp64():
    """hi*hi + hi*lo + lo*hi of two scaled columns reproduces their dot product to
    the split's accuracy (FP32 accumulation left out: the model sums in FP64)."""
    rng = np.random.Generator(np.random.PCG64(12))
    a = rng.standard_normal(2048) * 3.0
    b = rng.standard_normal(2048) * 1e-7
    sa, sb = 512.0, _colscale(float(np.max(np.abs(b))))
    ah, al = _split(a * sa)
    bh, bl = _split(b * sb)
    f = lambda u: u.astype(np.float64)
    dot = (np.dot(f(ah), f(bh)) + np.dot(f(ah), f(bl)) + np.dot(f(al), f(bh))) / (sa * sb)
    ref = float(np.dot(a, b))
    assert abs(dot - ref) <= 2.0 ** -20 * float(np.dot(np.abs(a), np.abs(b)))
