"""Pins for splitmix64 and for the quantizer / bit-plane packing."""

import os

import numpy as np
import pytest

from oracle import quant, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_published_outputs():
    expect = [int(l[0], 16) for l in _golden_lines("splitmix64.txt")]
    got = [int(x) for x in rng.stream(0, 4)]
    assert got == expect
    # counter-based: any window of the stream equals the same slice
    np.testing.assert_array_equal(rng.stream(12345, 5, start=3), rng.stream(12345, 8)[3:])


def test_uniform_pm1_range_and_exactness():
    u = rng.uniform_pm1(99, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0
    # every value is a multiple of 2^-52 (53-bit numerator times 2^-52 minus 1)
    assert np.all(((u + 1.0) * 2.0 ** 52) % 1.0 == 0.0)
    assert abs(u.mean()) < 0.01


def test_quantizer_endpoints_and_error_bound():
    x = np.random.default_rng(1).normal(size=(5, 1000))
    for bits in (1, 4, 12, 16):
        lo, hi = quant.quant_params(x, axis=1)
        s = quant.quantize(x, lo[:, None], hi[:, None], bits)
        assert s.min() >= 0 and s.max() <= (1 << bits) - 1
        amin = np.argmin(x, axis=1)
        amax = np.argmax(x, axis=1)
        assert np.all(s[np.arange(5), amin] == 0)
        assert np.all(s[np.arange(5), amax] == (1 << bits) - 1)
        xr = quant.dequantize(s, lo[:, None], hi[:, None], bits)
        step = (hi - lo) / ((1 << bits) - 1)
        assert np.all(np.abs(xr - x) <= step[:, None] * (0.5 + 1e-9))


def test_quantizer_constant_group_and_half_up():
    x = np.full(10, 2.5)
    s = quant.quantize(x, np.float64(2.5), np.float64(2.5), 12)
    assert np.all(s == 0)
    np.testing.assert_array_equal(quant.dequantize(s, 2.5, 2.5, 12), x)
    # exact ties round up: 3 levels on [0, 3] -> step 1, t = x exactly
    s = quant.quantize(np.array([0.5, 1.5, 2.5]), np.float64(0.0), np.float64(3.0), 2)
    np.testing.assert_array_equal(s, [1, 2, 3])


def test_pack_layout_by_hand():
    # 33 symbols of 3 bits: group 0 = symbols 0..31, group 1 = symbol 32 + padding
    s = np.zeros(33, dtype=np.int64)
    s[0] = 0b101       # bits 0 and 2 -> bit 0 of words 0 and 2
    s[31] = 0b010      # bit 1 -> bit 31 of word 1
    s[32] = 0b111      # group 1: bit 0 of words 3, 4, 5
    w = quant.pack_bits(s, 3)
    assert w.tolist() == [1, 1 << 31, 1, 1, 1, 1]
    np.testing.assert_array_equal(quant.unpack_bits(w, 3, 33), s)


@pytest.mark.parametrize("bits", [1, 5, 12, 16, 31])
def test_pack_roundtrip(bits):
    r = np.random.default_rng(bits)
    s = r.integers(0, 1 << bits, size=1000 + bits)
    w = quant.pack_bits(s, bits)
    assert w.shape[0] == quant.packed_words(s.shape[0], bits)
    np.testing.assert_array_equal(quant.unpack_bits(w, bits, s.shape[0]), s)
