"""Philox4x32-10 counter-based generator, written from its published definition.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (2011), Sec. 5 (the Philox S-box: two 32x32->64
multiplications per round, a Weyl sequence on the key, 10 rounds).

The paper's random states (Sec. II.A, Eqs. form1-form3 and Sec. III: random phases)
and Anderson disorder need a reproducible random source; the paper names none.
Both the oracle and the CUDA path draw from this generator, each with its own
implementation; they agree bit for bit because both follow the same published
definition, and this one is pinned to the published known-answer vectors.

Part of the FP64 oracle: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)


def philox4x32_10(ctr, key):
    """Apply 10 Philox rounds to the 4-word counter `ctr` under the 2-word key `key`.

    Each word may be a scalar or an integer array (broadcast together).  Returns a
    tuple of four uint32 arrays.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
        (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
    and the key then advances by the Weyl constants (W0, W1) mod 2^32.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK32 for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & _MASK32 for k in key)
    for _ in range(10):
        p0 = PHILOX_M0 * c0          # < 2^64: exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & _MASK32
        k1 = (k1 + PHILOX_W1) & _MASK32
    return tuple(np.asarray(v, dtype=np.uint32) for v in (c0, c1, c2, c3))


# Stream identifiers (third counter word).  Convention of this library:
#   counter = (index_lo, index_hi, stream, sub), key = (seed_lo, seed_hi)
STREAM_DISORDER = 0
STREAM_VACANCY = 1
STREAM_PHASE = 2


def draw_u32(seed: int, index, stream: int, sub: int = 0) -> np.ndarray:
    """First output word of Philox4x32-10 at counter (index, stream, sub) under `seed`."""
    index = np.asarray(index, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    out = philox4x32_10(
        (index & _MASK32, index >> _SHIFT32, np.uint64(stream), np.uint64(sub)),
        (np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)))
    return out[0]
