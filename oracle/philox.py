"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), written from its published definition.  Oracle side; the CUDA library carries its own
implementation of the same published generator.

One call maps a 128-bit counter (four 32-bit words) and a 64-bit key (two words) to four
32-bit outputs through ten rounds.  A round multiplies counter words 0 and 2 by the two Philox
multipliers, keeps the high and low halves, and mixes them with words 1 and 3 and the key; the
key is bumped by the two Weyl constants between rounds.

uniform53(): a double in [0, 1) from the first two output words (27 + 26 high bits).
"""
from __future__ import annotations

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def _round(c, k):
    p0 = M0 * c[0]
    p1 = M1 * c[2]
    hi0, lo0 = (p0 >> 32) & MASK, p0 & MASK
    hi1, lo1 = (p1 >> 32) & MASK, p1 & MASK
    return [(hi1 ^ c[1] ^ k[0]) & MASK, lo1, (hi0 ^ c[3] ^ k[1]) & MASK, lo0]


def philox4x32_10(ctr, key):
    c = [int(v) & MASK for v in ctr]
    k = [int(v) & MASK for v in key]
    for r in range(10):
        if r > 0:
            k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
        c = _round(c, k)
    return c


def uniform53(ctr, key) -> float:
    w = philox4x32_10(ctr, key)
    return ((w[0] >> 5) * 67108864.0 + (w[1] >> 6)) * (1.0 / 9007199254740992.0)


def key_of_seed(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return [seed & MASK, (seed >> 32) & MASK]
