"""Counter-based random numbers for the synthetic inputs.

The generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser is the one Vigna publishes
for seeding xoshiro).  SplitMix64 advances its state by a fixed odd constant and
returns a bijective mix of the state, so draw number c of a stream is
``mix(key + (c + 1) * GAMMA)``: any draw can be computed on its own, which lets
numpy produce whole arrays at once and keeps every draw a pure function of
(seed, stream, counter).

This module holds no N-body arithmetic.  It is shared, as input generation
only, by the oracle tests, the GPU tests and the benchmark.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)


def mix64(z):
    """SplitMix64 output function applied element-wise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of an independent stream: the mixed (seed, stream) pair."""
    with np.errstate(over="ignore"):
        k = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(stream))
    return np.uint64(k)


def u64(seed: int, stream: int, counter) -> np.ndarray:
    """Draws number ``counter`` (array of non-negative ints) of one stream."""
    c = np.asarray(counter, dtype=np.uint64)
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        return mix64(key + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, counter) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (u64(seed, stream, counter) >> _S11).astype(np.float64) * (2.0 ** -53)
