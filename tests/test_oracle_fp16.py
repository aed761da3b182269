"""Pins for the oracle's binary16 rounding (Section 1.2, Table 1).

The oracle's fl16 is written from the IEEE 754 round-to-nearest-even
definition on the double's bit pattern.  It is checked against numpy's
float16 conversion, an independent IEEE implementation, on every boundary
that a plausible mistake would move: each exact binary16 value, each midpoint
between neighbours (ties to even), one double ulp either side of each
midpoint, the subnormal range, the overflow boundary, plus random samples.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore:overflow encountered")


def _np16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def all_finite_halves():
    bits = np.arange(0, 0x10000, dtype=np.uint32).astype(np.uint16)
    h = bits.view(np.float16)
    return h[np.isfinite(h)].astype(np.float64)


def test_exact_halves_are_fixed_points():
    h = all_finite_halves()
    assert np.array_equal(O.fl16(h), h)


def test_midpoints_ties_to_even_and_neighbours():
    pos = np.unique(all_finite_halves()[all_finite_halves() >= 0])
    lo, hi = pos[:-1], pos[1:]
    mid = (lo + hi) / 2.0  # exact in double
    for probe in (mid, np.nextafter(mid, -np.inf), np.nextafter(mid, np.inf)):
        for s in (1.0, -1.0):
            got = O.fl16(s * probe)
            ref = _np16(s * probe)
            assert np.array_equal(got, ref), np.flatnonzero(got != ref)[:5]
    # ties: the even neighbour (last significand bit 0) wins
    even = (lo.astype(np.float16).view(np.uint16) & 1) == 0
    assert np.array_equal(O.fl16(mid), np.where(even, lo, hi))


def test_overflow_and_underflow_boundaries():
    assert O.fl16(65504.0) == 65504.0
    assert O.fl16(np.nextafter(65520.0, 0)) == 65504.0
    assert np.isinf(O.fl16(65520.0))  # tie between 65504 and 2^16 -> even -> inf
    assert np.isinf(O.fl16(1e10)) and O.fl16(-1e10) == -np.inf
    assert O.fl16(2.0 ** -25) == 0.0  # tie between 0 and 2^-24 -> 0
    assert O.fl16(np.nextafter(2.0 ** -25, 1)) == 2.0 ** -24
    assert O.fl16(2.0 ** -26) == 0.0
    assert O.fl16(3 * 2.0 ** -25) == 2.0 ** -23  # tie between 1 and 2 ulps -> even (2)
    assert O.fl16(2.0 ** -14) == 2.0 ** -14 and O.fl16(2.0 ** -24) == 2.0 ** -24
    assert np.isnan(O.fl16(np.nan))
    assert np.signbit(O.fl16(-1e-30))


def test_random_doubles_and_floats():
    g = np.random.default_rng(1)
    x = np.concatenate([
        g.standard_normal(200000) * 10.0 ** g.uniform(-9, 5, 200000),
        g.uniform(-70000, 70000, 100000),
        g.uniform(-2 ** -13, 2 ** -13, 100000),
    ])
    assert np.array_equal(O.fl16(x), _np16(x))
    f = x.astype(np.float32)
    assert np.array_equal(O.f16_bits_from_f32(f), f.astype(np.float16).view(np.uint16))


def test_bits_and_values_roundtrip():
    bits = np.arange(0, 0x10000, dtype=np.uint32).astype(np.uint16)
    h = bits.view(np.float16)
    fin = np.isfinite(h)
    got = np.array([O.lib().orc_f16_value(int(b)) for b in bits[fin][::97]])
    assert np.array_equal(got, h[fin][::97].astype(np.float64))
    got_bits = O.f16_bits_from_f32(h[fin].astype(np.float32))
    assert np.array_equal(got_bits, bits[fin])


def test_float32_patterns_strided():
    """Every 4099th float32 bit pattern (about 1e6 values spanning all
    exponents); the full 2^32 sweep runs with NL_SLOW=1."""
    bits = np.arange(0, 2 ** 32, 4099, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    assert np.array_equal(O.f16_bits_from_f32(f), f.astype(np.float16).view(np.uint16))


@pytest.mark.slow
def test_float32_patterns_exhaustive():
    for start in range(0, 2 ** 32, 2 ** 26):
        bits = np.arange(start, start + 2 ** 26, dtype=np.uint64).astype(np.uint32)
        f = bits.view(np.float32)
        f = f[np.isfinite(f)]
        assert np.array_equal(O.f16_bits_from_f32(f), f.astype(np.float16).view(np.uint16)), hex(start)
