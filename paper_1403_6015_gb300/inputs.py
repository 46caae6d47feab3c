"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This module holds no arithmetic of the HODLR method: it only draws points and right-hand
sides. Both the oracle and the CUDA path receive the arrays it produces, bit-identical.

Generator: splitmix64 in counter form (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). Element i of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15). Uniform doubles take the top 53 bits.
Normal deviates use the Box-Muller transform on two independent uniform streams.

The paper's workloads (Sec. 5) draw points uniformly in a cube and build C = s I + K on
them; the right-hand sides here are N(0, 1), so the log-likelihood is well defined.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return `count` uint64 outputs of the counter-form splitmix64 stream `seed`."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_points(n: int, d: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n points uniform in [lo, hi)^d, unsorted, as a C-contiguous (n, d) float64 array.

    Coordinate c of point i is element i*d + c of the stream, so the 1-D case is a
    plain vector of n draws.
    """
    u = uniform01(seed, n * d)
    return np.ascontiguousarray((lo + (hi - lo) * u).reshape(n, d))


def normal(n: int, seed: int, ncols: int = 1) -> np.ndarray:
    """N(0, 1) deviates by Box-Muller, shape (n,) for ncols == 1 else column-major (n, ncols).

    u1 lies in (0, 1] (one added to the 53-bit integer before scaling) so log(u1) is finite.
    """
    m = n * ncols
    z1 = splitmix64(seed, m)
    z2 = splitmix64(seed ^ 0x5DEECE66D, m)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    if ncols == 1:
        return g
    return np.asfortranarray(g.reshape(ncols, n).T)


# Workload recipes. Each returns (x, y) with x unsorted (n, d) and y (n,) or (n, nrhs).
# Seeds follow "1000 + workload index" for points and +1 for the right-hand side.

def workload_small_se(seed: int = 1000):
    """n=4096 points U[-1,1], y ~ N(0,1): the small squared-exponential case."""
    n = 4096
    return uniform_points(n, 1, -1.0, 1.0, seed), normal(n, seed + 1)


def workload_1d(n: int, seed: int, nrhs: int = 1, lo: float = -1.0, hi: float = 1.0):
    """n points U[lo,hi) in 1-D and nrhs N(0,1) right-hand sides."""
    return uniform_points(n, 1, lo, hi, seed), normal(n, seed + 1, nrhs)


def workload_2d(n: int, seed: int, nrhs: int = 1):
    """n points U[0,1)^2 and nrhs N(0,1) right-hand sides."""
    return uniform_points(n, 2, 0.0, 1.0, seed), normal(n, seed + 1, nrhs)


def workload_3d(n: int, seed: int, nrhs: int = 1):
    """n points U[0,1)^3 and nrhs N(0,1) right-hand sides."""
    return uniform_points(n, 3, 0.0, 1.0, seed), normal(n, seed + 1, nrhs)
