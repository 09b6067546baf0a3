"""Uniform scalar quantizer Q(.) and bit-plane packing.

Test infrastructure (see ``oracle/__init__``).

The paper names a quantization function Q(.) (Eq. 10, Eq. 12) but does not
define it; it assumes 16 bits per dictionary element and per anchor
coordinate (Section IV, before Eq. 13).  The codec's reading:

* Per group of values (a row of the coefficient matrix, a column of the
  dictionary, all anchor values of one coordinate): lo = min, hi = max,
  range = hi - lo, scale = (2^b - 1) / range (one correctly rounded
  division; scale = 0 when range == 0).
* Symbol: t = (x - lo) * scale with the subtraction and the product rounded
  separately (no fused multiply-add), s = floor(t + 0.5) (round half up),
  clamped to [0, 2^b - 1].
* Reconstruction: step = range / (2^b - 1); x_hat = lo + s * step (again no
  fused multiply-add).
* b = 0 means "no quantization": the raw binary64 values are stored.

Packing: symbols are taken in groups of 32.  For group g of a b-bit
section, 32-bit word g*b + j holds bit j of symbols 32g .. 32g+31, symbol
32g + l in bit l (one bit plane per word).  The last group is padded with
zero symbols.  Words are little-endian.

Pinned by: lo -> 0, hi -> 2^b - 1, |x - x_hat| <= step/2 (+ rounding),
constant groups, and pack/unpack round trips (tests/test_oracle_quant.py).
The quantizer itself is a convention the paper leaves open: parity
unpinned beyond these properties.
"""

import numpy as np


def quant_params(x, axis=None):
    lo = np.min(x, axis=axis)
    hi = np.max(x, axis=axis)
    return np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)


def quantize(x, lo, hi, bits):
    """x, lo, hi broadcastable float64 arrays -> int64 symbols."""
    levels = float((1 << bits) - 1)
    rng_ = np.asarray(hi - lo, dtype=np.float64)
    with np.errstate(divide="ignore"):
        scale = np.where(rng_ > 0, levels / np.where(rng_ > 0, rng_, 1.0), 0.0)
    t = (x - lo) * scale
    s = np.floor(t + 0.5)
    s = np.clip(s, 0.0, levels)
    return s.astype(np.int64)


def dequantize(s, lo, hi, bits):
    levels = float((1 << bits) - 1)
    step = (hi - lo) / levels
    return lo + s.astype(np.float64) * step


def pack_bits(symbols, bits):
    """int symbols (1-D) -> uint32 words (bit-plane layout above)."""
    s = np.asarray(symbols, dtype=np.uint64).ravel()
    G = (s.shape[0] + 31) // 32
    padded = np.zeros(G * 32, dtype=np.uint64)
    padded[: s.shape[0]] = s
    padded = padded.reshape(G, 32)
    shifts = np.arange(32, dtype=np.uint64)
    words = np.zeros((G, bits), dtype=np.uint64)
    for j in range(bits):
        plane = (padded >> np.uint64(j)) & np.uint64(1)
        words[:, j] = (plane << shifts[None, :]).sum(axis=1)
    return words.astype(np.uint32).ravel()


def unpack_bits(words, bits, count):
    w = np.asarray(words, dtype=np.uint64).reshape(-1, bits)
    G = w.shape[0]
    shifts = np.arange(32, dtype=np.uint64)
    s = np.zeros((G, 32), dtype=np.uint64)
    for j in range(bits):
        plane = (w[:, j][:, None] >> shifts[None, :]) & np.uint64(1)
        s |= plane << np.uint64(j)
    return s.ravel()[:count].astype(np.int64)


def packed_words(count, bits):
    return ((count + 31) // 32) * bits
