"""Counter-based random numbers for the synthetic workloads.

The generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter form: the i-th
draw of a stream is the SplitMix64 output function applied to
``key + (i + 1) * GOLDEN``.  Every draw is therefore addressable by
(seed, stream, index) and the same numbers come out on any machine.

These numbers are *inputs*: edge weights, random start vectors, right-hand
sides.  Nothing here knows about Laplacians, trees or the sparsification
method; the same arrays are handed to the CPU checker and to the GPU library.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers used by the workload recipes
STREAM_WEIGHTS = 1
STREAM_EXTRA = 2      # chords, vias, Chung-Lu endpoints
STREAM_PADS = 3       # diagonal loads D
STREAM_RHS = 300      # right-hand side b of the SDD solve
STREAM_H0 = 1000      # + round: embedding start block
STREAM_V0 = 2000      # + round: lambda_max start vector


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(s ^ _mix(t + GOLDEN))[0]


def raw64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of (seed, stream) as uint64."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(key + idx * GOLDEN)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    x = raw64(seed, stream, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform (cosine branch).

    Draw k uses uniforms 2k and 2k+1 of the stream.
    """
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_block(seed: int, stream: int, n: int, r: int) -> np.ndarray:
    """n x r row-major block of N(0,1) draws; entry (i, j) is draw i*r + j."""
    return normal(seed, stream, n * r).reshape(n, r)
