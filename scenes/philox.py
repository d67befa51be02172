"""Philox4x32-10 counter-based generator written with torch int64 tensor ops.

Definition: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11 (the Philox-4x32 bijection, 10 rounds, with the multipliers
and Weyl key increments given there).  Every draw is a pure function of its
128-bit counter and 64-bit key, so a frame can be regenerated on any device
and in any order.

Products of two 32-bit words do not fit a signed int64, so the multiplier's
operand is split into 16-bit halves and the high/low words are reassembled
from two 48-bit partial products.
"""
from __future__ import annotations

import torch

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def _mulhilo(m: int, b: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """(hi, lo) 32-bit words of the 64-bit product m*b, m constant, b in [0, 2^32)."""
    bl = b & 0xFFFF
    bh = b >> 16
    p1 = bl * m                       # < 2^48
    p2 = bh * m                       # < 2^48
    lo = (((p2 & 0xFFFF) << 16) + p1) & _MASK32
    hi = (p2 + (p1 >> 16)) >> 16
    return hi & _MASK32, lo


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Apply Philox4x32-`rounds` to counters (int64 tensors holding uint32 values).

    Returns the four output words as int64 tensors in [0, 2^32).
    """
    k0 &= _MASK32
    k1 &= _MASK32
    for r in range(rounds):
        hi0, lo0 = _mulhilo(_M0, c0)
        hi1, lo1 = _mulhilo(_M1, c2)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        if r + 1 < rounds:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
    return c0, c1, c2, c3


def uniform_open01(words: torch.Tensor) -> torch.Tensor:
    """Map uint32 words to float64 uniforms strictly inside (0, 1): (x + 1/2) / 2^32."""
    return (words.to(torch.float64) + 0.5) * (1.0 / 4294967296.0)
