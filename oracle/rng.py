"""Counter-based random numbers for the oracle.

splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: the value for
counter i under seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).  Uniform
doubles use the top 53 bits; normals use the Box-Muller transform on two
consecutive counters.  The GPU library implements the same published
definition independently.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """mix(seed + (counter + 1) * golden) for an array of uint64 counters."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    return ((splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def normal_block(seed: int, n: int, b: int, offset: int = 0) -> np.ndarray:
    """n x b i.i.d. N(0,1) block; element (i, c) uses counters 2k, 2k+1 with k = offset + i*b + c."""
    k = np.arange(n * b, dtype=np.uint64) + np.uint64(offset)
    u1 = uniform01(seed, 2 * k)
    u2 = uniform01(seed, 2 * k + 1)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(n, b)
