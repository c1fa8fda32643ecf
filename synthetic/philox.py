"""Counter-based random numbers: Philox4x32-10 and Box-Muller normals.

Philox4x32-10 is the generator published by Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter is
scrambled by ten rounds of two 32x32->64-bit multiplies with a Weyl-sequence
key schedule.  Everything here is integer arithmetic on numpy uint64 arrays,
so the bit stream is identical on every platform.  Normal deviates come from
the Box-Muller transform of pairs of uniforms in the open interval (0, 1).

This module only makes seeded synthetic inputs; it holds none of the
filter's arithmetic.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply ten Philox rounds to counters (c0..c3) under key (k0, k1).

    All arguments broadcast; they are taken modulo 2**32.  Returns four
    uint64 arrays holding 32-bit words.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def uint32_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` 32-bit words of stream `stream` under `seed`, starting at word `offset`.

    Block i (four words) uses counter (i mod 2**32, i >> 32, stream, 0) and
    key (seed mod 2**32, seed >> 32).
    """
    if count <= 0:
        return np.zeros(0, dtype=np.uint64)
    first = offset // 4
    last = (offset + count + 3) // 4
    i = np.arange(first, last, dtype=np.uint64)
    w = philox4x32_10(i & _MASK, i >> _S32, np.uint64(stream), np.uint64(0),
                      np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    words = np.stack(w, axis=1).reshape(-1)
    start = offset - first * 4
    return words[start:start + count]


def uniform_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform deviates (w + 1/2) / 2**32 in the open interval (0, 1), float64."""
    w = uint32_stream(seed, stream, count, offset)
    return (w.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def normal_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller on consecutive uniform pairs.

    Normal 2t uses sqrt(-2 ln u_2t) cos(2 pi u_2t+1), normal 2t+1 the sine;
    `offset` counts normals and must be even.
    """
    if offset % 2:
        raise ValueError("normal_stream offset must be even")
    npair = (count + 1) // 2
    u = uniform_stream(seed, stream, 2 * npair, 2 * offset // 2).reshape(npair, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = (2.0 * np.pi) * u[:, 1]
    z = np.empty((npair, 2), dtype=np.float64)
    z[:, 0] = rad * np.cos(ang)
    z[:, 1] = rad * np.sin(ang)
    return z.reshape(-1)[:count]
