"""PRN sequences from a linear feedback shift register, and their circulant (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU baseline of
the benchmark.

Sec. 4 names a circulant built on a pseudo-random-noise signal that a linear feedback shift
register produces (``LFSRCirculant``) without giving the register's conventions.  Reading
used here (a Fibonacci register): an nbits-bit state s (nonzero), a tap mask T; each step
outputs o = s & 1, forms the feedback f = parity(s & T) and shifts s <- (s >> 1) |
(f << (nbits - 1)).  The circulant's first column holds c[k] = 1 - 2 o_k (bit 0 -> +1,
bit 1 -> -1) for the first n outputs.  The taps of x^m + x^a + 1 are bits 0 and a, which
gives the recurrence s_{k+m} = s_k xor s_{k+a}.

Pinned by tests/test_oracle_pins.py: a hand-stepped 3-bit register and the textbook
properties of maximal-length sequences (period 2^m - 1, 2^(m-1) ones per period, periodic
autocorrelation -1 of the +-1 sequence at every nonzero shift).
"""
from __future__ import annotations

import numpy as np

from .operators import Circulant


def lfsr_bits(nbits: int, taps: int, state: int, n: int) -> np.ndarray:
    if not 1 <= nbits <= 63 or state == 0 or state >> nbits:
        raise ValueError("state must be a nonzero nbits-bit value")
    out = np.empty(n, dtype=np.int64)
    s = state
    for k in range(n):
        out[k] = s & 1
        f = bin(s & taps).count("1") & 1
        s = (s >> 1) | (f << (nbits - 1))
    return out


def lfsr_sequence(nbits: int, taps: int, state: int, n: int) -> np.ndarray:
    """c[k] = 1 - 2 o_k for the first n output bits."""
    return 1.0 - 2.0 * lfsr_bits(nbits, taps, state, n)


def LFSRCirculant(nbits: int, taps: int, state: int, n: int) -> Circulant:
    return Circulant(lfsr_sequence(nbits, taps, state, n))
