"""Seeded synthetic operands shared by the tests, the smoke check and the bench.

This module holds none of the multiplication method's arithmetic: it only
draws bits.  Both the CUDA path's callers and the oracle's callers take their
inputs from here, so the two sides see the same operands.

Generator: SplitMix64 in counter form, word i of a stream = mix(seed + (i+1) * gamma)
with gamma = 0x9E3779B97F4A7C15 and the published SplitMix64 finaliser.

Workload shape (the paper times products of random bit-polynomials of
power-of-two lengths, Sec. 5.1): uniform random bits packed little-endian
into uint64 words (bit t of word w is the coefficient of x^(64 w + t)).  The
bits at and above the operand length in the last word are filled with
garbage by default, so that callers exercise tail masking.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 0x18031130


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` words of the SplitMix64 stream ``seed``, starting at word ``offset``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def config_seed(config: int, index: int) -> int:
    """Seed of product ``index`` of workload ``config`` (1-based config numbers)."""
    return BASE_SEED + 1000 * config + index


def operand(seed: int, nbits: int, garbage_tail: bool = True, top_bit: bool = False) -> np.ndarray:
    """A random nbits-bit polynomial as ceil(nbits/64) uint64 words.

    ``garbage_tail``: fill the bits >= nbits of the last word with random bits
    (they are not part of the operand).  ``top_bit``: force the coefficient of
    x^(nbits-1) to 1 so that the degree is exactly nbits-1.
    """
    nw = (nbits + 63) // 64
    w = splitmix64(seed, nw)
    r = nbits % 64
    if nw and not garbage_tail and r:
        w[-1] &= np.uint64((1 << r) - 1)
    if nw and top_bit:
        w[(nbits - 1) // 64] |= np.uint64(1 << ((nbits - 1) % 64))
    return w


def mask_tail(words: np.ndarray, nbits: int) -> np.ndarray:
    """Copy of ``words`` with every bit at or above ``nbits`` cleared."""
    w = np.array(words, dtype=np.uint64, copy=True)
    nw = (nbits + 63) // 64
    w[nw:] = 0
    if nbits % 64 and nw:
        w[nw - 1] &= np.uint64((1 << (nbits % 64)) - 1)
    return w


def loguniform_lengths(seed: int, count: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """floor(2^U) with U uniform on [lo_exp, hi_exp), one per product (int64)."""
    u = splitmix64(seed, count).astype(np.float64) / float(1 << 64)
    return np.floor(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the stream ``seed`` (53-bit resolution)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
