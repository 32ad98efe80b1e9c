"""Counter-based random numbers for the synthetic inputs.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i (1-based) of a stream with seed s is
mix(s + i * 0x9E3779B97F4A7C15) with the published finaliser constants.
Normals use the Box-Muller transform in float64.  Everything is vectorised
numpy; the arrays are cast to float32 once by the callers, so the oracle and
the CUDA path read identical float32 inputs.

This module holds no arithmetic of the rendering method.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a(name: str) -> int:
    h = 0xCBF29CE484222325
    for b in name.encode():
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def stream_seed(seed: int, name: str) -> np.uint64:
    """Derive an independent stream seed from a user seed and a stream name."""
    with np.errstate(over="ignore"):
        z = np.array([(seed * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        z ^= np.uint64(_fnv1a(name))
        return _mix(z)[0]


def splitmix64(seed: np.uint64, n: int) -> np.ndarray:
    """First n outputs of the SplitMix64 stream with the given seed (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        return _mix(np.uint64(seed) + i * _GOLDEN)


class Stream:
    """A named SplitMix64 stream; successive draws continue the counter."""

    def __init__(self, seed: int, name: str):
        self.seed = stream_seed(seed, name)
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            i = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
            out = _mix(self.seed + i * _GOLDEN)
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Uniform float64 in [lo, hi) from the top 53 bits."""
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def uniform_open0(self, n: int) -> np.ndarray:
        """Uniform float64 in (0, 1]."""
        return ((self.bits(n) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)

    def normal(self, n: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
        """Box-Muller normals, float64."""
        m = (n + 1) // 2
        u1 = self.uniform_open0(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m, dtype=np.float64)
        z[0::2] = r * np.cos(2.0 * np.pi * u2)
        z[1::2] = r * np.sin(2.0 * np.pi * u2)
        return mean + std * z[:n]

    def log_uniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.exp(self.uniform(n, np.log(lo), np.log(hi)))
