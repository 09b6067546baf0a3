"""splitmix64, written from its published definition.

Test infrastructure (see ``oracle/__init__``).

Output i (i = 0, 1, ...) of a generator seeded with ``s`` is
``mix(s + (i + 1) * GAMMA mod 2**64)`` where ``mix`` is the finaliser
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as in Vigna's public-domain C version).
Because output i depends only on (s, i) the generator is counter based and
both the oracle and the CUDA path can draw any element independently.

Pinned by the published first outputs for seed 0 (tests/golden/splitmix64.txt).

Uses in the codec (salts are part of the codec's definition):

* anchor keys:   seed ^ ANCHOR_SALT, element i = vertex i
* start basis:   seed ^ (BASIS_SALT + c) for coordinate c, element f*k + j
"""

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
ANCHOR_SALT = 0x616E63686F727321   # ASCII "anchors!"
BASIS_SALT = 0x62617369735F3030    # ASCII "basis_00"


def _mix(z):
    """splitmix64 finaliser on a uint64 numpy array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream(seed, count, start=0):
    """Outputs start .. start+count-1 of splitmix64 seeded with ``seed``."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
    return _mix(state)


def uniform_pm1(seed, count):
    """Doubles in [-1, 1): top 53 bits scaled by 2**-53, times 2, minus 1.

    Every step is exact in binary64, so both sides get identical values.
    """
    u = stream(seed, count) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
