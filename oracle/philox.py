"""Oracle: Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The EA of Appendix A draws all its random numbers from this generator, on the device and in
the oracle alike, so the two sides see the same numbers for the same (key, counter). This is a
plain restatement of the published definition: ten rounds, each multiplying words 0 and 2 by
the round multipliers (full 128-bit products), and the key bumped by the Weyl constants
between rounds.

Pinned by tests/test_oracle_philox.py against numpy's own Philox bit generator (an independent
implementation of the same definition) and against the published known-answer vector for
counter 0, key 0.

Draw conventions shared with the device (each is a plain definition, not a transform of the
method):
* ``u01(x)``            = (x >> 11) * 2^-53, a double in [0, 1);
* ``uniform_int(x, n)`` = ((x >> 32) * n) >> 32, an integer in [0, n);
* ``bit(x)``            = x >> 63.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
ROUNDS = 10
_MASK = (1 << 64) - 1


def philox4x64_scalar(counter, key, rounds=ROUNDS):
    """One block of four 64-bit words, with Python integers (reference form of the definition)."""
    x = [int(c) & _MASK for c in counter]
    k = [int(v) & _MASK for v in key]
    for r in range(rounds):
        if r:
            k = [(k[0] + W0) & _MASK, (k[1] + W1) & _MASK]
        p0 = M0 * x[0]
        p1 = M1 * x[2]
        x = [(p1 >> 64) ^ x[1] ^ k[0], p1 & _MASK, (p0 >> 64) ^ x[3] ^ k[1], p0 & _MASK]
    return x


def _mulhilo(a, m):
    """128-bit product of uint64 arrays a and the constant m, as (hi, lo) uint64 arrays."""
    lo32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    m_lo, m_hi = np.uint64(m & 0xFFFFFFFF), np.uint64(m >> 32)
    a_lo, a_hi = a & lo32, a >> s32
    ll = a_lo * m_lo
    lh = a_lo * m_hi
    hl = a_hi * m_lo
    hh = a_hi * m_hi
    mid = (ll >> s32) + (lh & lo32) + (hl & lo32)
    lo = (mid << s32) | (ll & lo32)
    hi = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    return hi, lo


def philox4x64(c0, c1, c2, c3, key0, key1, rounds=ROUNDS):
    """Vectorised Philox4x64: counter words and key words broadcast; returns (..., 4) uint64."""
    with np.errstate(over="ignore"):
        x = [np.asarray(c, dtype=np.uint64) for c in np.broadcast_arrays(c0, c1, c2, c3)]
        k0 = np.uint64(int(key0) & _MASK)
        k1 = np.uint64(int(key1) & _MASK)
        for r in range(rounds):
            if r:
                k0 = np.uint64((int(k0) + W0) & _MASK)
                k1 = np.uint64((int(k1) + W1) & _MASK)
            hi0, lo0 = _mulhilo(x[0], M0)
            hi1, lo1 = _mulhilo(x[2], M1)
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
        return np.stack(x, axis=-1)


def u01(x):
    """Double in [0, 1) from the top 53 bits of a 64-bit word."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_int(x, n):
    """Integer in [0, n) from the top 32 bits of a 64-bit word (n < 2^31)."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)


def bit(x):
    """Top bit of a 64-bit word, 0 or 1."""
    return np.asarray(x, dtype=np.uint64) >> np.uint64(63)
