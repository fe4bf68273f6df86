"""Counter-based SplitMix64 streams (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).

SplitMix64 advances a 64-bit state by the golden-ratio increment
0x9E3779B97F4A7C15 and returns a bijective mix of the new state. Because the
state after k steps is simply ``seed + k * gamma`` (mod 2**64), element k of a
stream can be computed on its own, which makes the generator counter-based:
the vectorised form below produces the same numbers as stepping one value at
a time.

This module draws random numbers only. It holds none of the reconstruction
method's arithmetic; both the CUDA library's tests/bench and the FP64 oracle
take their random inputs from here.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the stream started at ``seed``.

    Output k is ``mix64(seed + (k + 1) * gamma)``, i.e. the value returned by
    the (k+1)-th call of the sequential generator.
    """
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & _MASK64) + k * GAMMA
    return mix64(state)


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each output."""
    return (u64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by the Box-Muller transform (Box & Muller, 1958).

    Pair p uses uniforms 2p and 2p+1 of the stream: u1 is mapped to (0, 1]
    so the logarithm is finite; the pair yields r*cos(2*pi*u2) and
    r*sin(2*pi*u2). ``offset`` counts normals and must be even, so that a
    stream drawn in chunks equals the stream drawn at once.
    """
    if offset % 2:
        raise ValueError("normal(): offset must be even")
    npairs = (n + 1) // 2
    u = uniform(seed, 2 * npairs, offset)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npairs)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]


def derive(seed: int, *tags: int) -> int:
    """A child seed: the stream of ``seed`` folded with integer tags."""
    s = np.uint64(seed & _MASK64)
    for t in tags:
        with np.errstate(over="ignore"):
            s = mix64(np.uint64((int(s) ^ (t & _MASK64)) & _MASK64) + GAMMA)
    return int(s)
