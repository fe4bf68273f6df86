"""Minibatch index sampler (Sec. III): each step draws |Omega| projection
indices at random from the MN pixels; one epoch is ceil(MN/|Omega|) steps.

Construction (this library's choice; the paper does not say how the random
subsets are drawn): every epoch e uses a keyed bijection pi_e of [0, MN),
so that an epoch visits every pixel. Step s is epoch e = s div spe with
spe = ceil(MN/B) and position j = s mod spe in it; its slot b takes
pi_e((j*B + b) mod MN). The last step of an epoch therefore wraps to the
start of the same permutation.

pi_e is a 4-round balanced Feistel network on 2*h bits (h = ceil(bits/2),
bits = max(2, ceil(log2 MN))) with round function F(R, k) = mix64(R xor k)
mod 2^h, where mix64 is the SplitMix64 output function and round key r of
epoch e is output 4e + r of the SplitMix64 stream of the sampler seed (Luby &
Rackoff 1988 for the Feistel bijection; Black & Rogaway 2002 for cycle
walking, which maps a bijection of [0, 2^2h) onto [0, MN) by re-applying it
until the value lands below MN).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _mix64(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def half_bits(n: int) -> int:
    bits = max(2, (n - 1).bit_length())
    return (bits + 1) // 2


def round_keys(seed: int, epoch: int):
    return [_mix64(seed + (4 * epoch + r + 1) * _GAMMA) for r in range(4)]


def feistel(x: int, keys, h: int) -> int:
    mask = (1 << h) - 1
    L, R = x >> h, x & mask
    for k in keys:
        L, R = R, L ^ (_mix64(R ^ k) & mask)
    return (L << h) | R


def permute(x: int, n: int, seed: int, epoch: int) -> int:
    """pi_e(x) for x in [0, n), by cycle walking."""
    h = half_bits(n)
    keys = round_keys(seed, epoch)
    y = feistel(x, keys, h)
    while y >= n:
        y = feistel(y, keys, h)
    return y


def steps_per_epoch(B: int, n: int) -> int:
    """ceil(n / B) steps of B rays make one epoch over n pixels."""
    return -(-n // B)


def epoch_of(step: int, B: int, n: int) -> int:
    """The epoch (0-based) that training step `step` (0-based) falls in."""
    return step // steps_per_epoch(B, n)


def minibatch(step: int, B: int, n: int, seed: int) -> np.ndarray:
    """The B indices of training step `step` (0-based)."""
    e, j = divmod(step, steps_per_epoch(B, n))
    return np.array([permute((j * B + b) % n, n, seed, e) for b in range(B)],
                    dtype=np.int64)
