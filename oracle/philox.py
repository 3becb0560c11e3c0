"""Philox4x32-10 counter-based random numbers (oracle side).

Written from the published definition: J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11 -- a 10-round
Feistel-like bijection of a 128-bit counter under a 64-bit key, each round
multiplying two counter words by fixed 32-bit multipliers and xoring the high
halves with the other words and the key; the key is advanced by two Weyl
constants between rounds.

The product implements the same published generator independently in CUDA and
C++; the two share no code. Test infrastructure only.

Works element-wise on Python ints or on numpy uint64 arrays that hold 32-bit
values.
"""
import numpy as np

_MUL0 = 0xD2511F53
_MUL1 = 0xCD9E8D57
_WEYL0 = 0x9E3779B9
_WEYL1 = 0xBB67AE85
_M32 = 0xFFFFFFFF

# purpose words (third counter word) that separate the random streams
PURPOSE_TRACK = 1
PURPOSE_NOISE = 2
PURPOSE_INIT = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counter (c0..c3) and key (k0, k1)."""
    as_np = any(isinstance(v, np.ndarray) for v in (c0, c1, c2, c3, k0, k1))
    if as_np:
        c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & np.uint64(_M32)
                                  for v in (c0, c1, c2, c3, k0, k1))
        m32 = np.uint64(_M32)
        mul0, mul1 = np.uint64(_MUL0), np.uint64(_MUL1)
        weyl0, weyl1 = np.uint64(_WEYL0), np.uint64(_WEYL1)
        s32 = np.uint64(32)
    else:
        m32, mul0, mul1, weyl0, weyl1, s32 = _M32, _MUL0, _MUL1, _WEYL0, _WEYL1, 32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + weyl0) & m32
            k1 = (k1 + weyl1) & m32
        p0 = mul0 * c0          # < 2**64: exact in uint64 and in Python ints
        p1 = mul1 * c2
        hi0, lo0 = p0 >> s32, p0 & m32
        hi1, lo1 = p1 >> s32, p1 & m32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m32, lo1, (hi0 ^ c3 ^ k1) & m32, lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Key words of a 64-bit seed: (low 32 bits, high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & _M32, seed >> 32


def uniform01(lo_word, hi_word):
    """U[0,1) double from 64 random bits (lo | hi << 32): top 53 bits times 2**-53."""
    u = int(lo_word) | (int(hi_word) << 32)
    return float(u >> 11) * (2.0 ** -53)


def draw(seed, purpose, obj, var, event=0):
    """Two independent U[0,1) doubles for (object, variate) of a purpose stream."""
    k0, k1 = seed_key(seed)
    w0, w1, w2, w3 = philox4x32_10(obj, var, purpose, event, k0, k1)
    return uniform01(w0, w1), uniform01(w2, w3)
