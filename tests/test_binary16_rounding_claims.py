"""The arithmetic claims the binary16 kernels rest on, checked on the CPU with
numpy's IEEE float16/float32/float64 (an implementation independent of both
the CUDA path and the oracle):

* the product of two binary16 numbers is exact in binary32, so rounding it
  once to binary16 is the correctly rounded binary16 product;
* a difference or a quotient of two binary16 numbers formed in binary32 and
  then rounded to binary16 equals the one formed in binary64 and rounded to
  binary16 (the correctly rounded result in both cases: 24 and 53 are both at
  least 2 * 11 + 2).

The binary16-arithmetic LU and triangular solves form their products,
differences and quotients this way; the oracle forms them in binary64."""
import numpy as np


def _all_finite_halves():
    h = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16).view(np.float16)
    return h[np.isfinite(h)]


def _pairs(n, seed):
    g = np.random.default_rng(seed)
    h = _all_finite_halves()
    a = h[g.integers(0, h.size, n)]
    b = h[g.integers(0, h.size, n)]
    # and pairs whose exponents are close (the cancelling differences)
    c = h[g.integers(0, h.size, n)]
    with np.errstate(over="ignore"):
        d = (c.astype(np.float32) * (1.0 + g.uniform(-1e-2, 1e-2, n)).astype(np.float32)).astype(np.float16)
    return np.concatenate([a, c]), np.concatenate([b, d])


def test_binary16_product_exact_in_binary32():
    a, b = _pairs(1_000_000, 1)
    with np.errstate(over="ignore"):
        p32 = a.astype(np.float32) * b.astype(np.float32)
        p64 = a.astype(np.float64) * b.astype(np.float64)
        r32, r64 = p32.astype(np.float16), p64.astype(np.float16)
    assert np.array_equal(p32.astype(np.float64), p64)  # exact: 11 + 11 bits
    assert np.array_equal(r32, r64)


def test_binary16_difference_through_binary32_is_correctly_rounded():
    a, b = _pairs(2_000_000, 2)
    with np.errstate(over="ignore", invalid="ignore"):
        via32 = (a.astype(np.float32) - b.astype(np.float32)).astype(np.float16)
        via64 = (a.astype(np.float64) - b.astype(np.float64)).astype(np.float16)  # the double difference is exact
    same = (via32 == via64) | (np.isnan(via32) & np.isnan(via64))
    assert same.all(), (a[~same][:5], b[~same][:5])


def test_binary16_quotient_through_binary32_is_correctly_rounded():
    a, b = _pairs(2_000_000, 3)
    keep = b != 0
    a, b = a[keep], b[keep]
    with np.errstate(over="ignore", invalid="ignore", under="ignore"):
        via32 = (a.astype(np.float32) / b.astype(np.float32)).astype(np.float16)
        via64 = (a.astype(np.float64) / b.astype(np.float64)).astype(np.float16)
    same = (via32 == via64) | (np.isnan(via32) & np.isnan(via64))
    assert same.all(), (a[~same][:5], b[~same][:5])


def test_binary16_difference_all_pairs_of_one_exponent_band():
    """Exhaustive over all finite binary16 a and every b from a band of 512
    values around 1 (the band where the pivots of the H-equation Jacobian
    live), including the subnormal results of near-cancellation."""
    h = _all_finite_halves()
    band = np.arange(0x3a00, 0x3c00, dtype=np.uint16).view(np.float16)
    a = np.repeat(h, band.size)
    b = np.tile(band, h.size)
    with np.errstate(over="ignore", invalid="ignore"):
        via32 = (a.astype(np.float32) - b.astype(np.float32)).astype(np.float16)
        via64 = (a.astype(np.float64) - b.astype(np.float64)).astype(np.float16)
        q32 = (a.astype(np.float32) / b.astype(np.float32)).astype(np.float16)
        q64 = (a.astype(np.float64) / b.astype(np.float64)).astype(np.float16)
    assert np.array_equal(via32, via64)
    assert np.array_equal(q32, q64)
