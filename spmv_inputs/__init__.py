"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and nothing else: it holds none of the
SpMV, compression or CG arithmetic.  Both the CUDA path and the CPU oracle
receive the arrays it returns, so neither side generates its own vectors.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  One step adds the golden gamma
0x9E3779B97F4A7C15 to the 64-bit state and returns the state passed through
the mix  z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
z *= 0x94D049BB133111EB; z ^= z>>31.  Step k (k = 1, 2, ...) of a stream
started at state s0 therefore outputs mix(s0 + k*gamma), which lets numpy
draw a whole stream at once.

Independent purposes use independent streams: the starting state of the
stream for (seed, tag) is the first output of a SplitMix64 started at
seed XOR tag, where tag is the purpose name's ASCII bytes read as a
little-endian integer ("x", "drop", "special", "val", "perm", "grid").
A uniform double in [0, 1) is (next >> 11) * 2**-53; U[lo, hi) is
lo + (hi - lo) * u, evaluated in IEEE double.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def tag_value(tag: str) -> int:
    """The purpose name's ASCII bytes as a little-endian unsigned integer."""
    return int.from_bytes(tag.encode("ascii"), "little") & MASK64


def _mix_scalar(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_next(state: int) -> tuple[int, int]:
    """One SplitMix64 step: returns (new_state, output)."""
    state = (state + GAMMA) & MASK64
    return state, _mix_scalar(state)


def stream_state(seed: int, tag: str) -> int:
    """Starting state of the independent stream for (seed, tag)."""
    _, out = splitmix64_next((seed ^ tag_value(tag)) & MASK64)
    return out


def splitmix64_block(state: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs number start+1 .. start+count of the stream whose state is `state`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state) + k * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(state: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) with 53 random bits each."""
    z = splitmix64_block(state, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, tag: str = "x") -> np.ndarray:
    """x_i ~ U[lo, hi) in index order, float64, from the (seed, tag) stream."""
    u = uniform01(stream_state(seed, tag), n)
    return lo + (hi - lo) * u


def uniform_matrix(n: int, k: int, seed: int, lo: float = -1.0, hi: float = 1.0, tag: str = "x") -> np.ndarray:
    """An n x k row-major float64 block drawn in row-major order."""
    return uniform_vector(n * k, seed, lo, hi, tag).reshape(n, k)


def integer_vector(n: int, seed: int, lo: int = -3, hi: int = 3, tag: str = "x") -> np.ndarray:
    """Integers in [lo, hi] as float64 (every partial sum of A x is then exact)."""
    u = uniform01(stream_state(seed, tag), n)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.float64)


def grid_edges(count: int, seed: int, lo: int = 16, hi: int = 96, tag: str = "grid") -> list[int]:
    """count grid edge lengths drawn uniformly from the integers lo..hi inclusive."""
    u = uniform01(stream_state(seed, tag), count)
    return [int(lo + np.floor(v * (hi - lo + 1))) for v in u]


# Workload shapes of the paper's HPCG experiment and its variants, by name.
WORKLOADS = {
    "hpcg_32": dict(nx=32, ny=32, nz=32, x_seed=0),
    "hpcg_192": dict(nx=192, ny=192, nz=192, x_seed=1),
    "irregular_128": dict(nx=128, ny=128, nz=128, seed=2, x_seed=2),
    "hpcg_160_spmm": dict(nx=160, ny=160, nz=160, x_seed=3, ks=(1, 4, 8, 16, 32)),
    "ragged_24": dict(count=24, seed=4, lo=16, hi=96),
}
