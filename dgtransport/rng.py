"""Counter-based random numbers (splitmix64) for seeded synthetic inputs.

Every random draw in the synthetic transport problems (vertex jitter, the
log-normal absorption, the functional weights of the adjoint check) comes from
this generator, so a problem is identical on every machine and in every
process.  splitmix64 is Steele, Lea and Flood's 64-bit mixer (OOPSLA 2014):
the i-th output for a given seed is a pure function of (seed, i).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, index):
    """Return the splitmix64 output for counter ``index`` (array) under ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, stream=0):
    """``n`` doubles in [0, 1) from 53 high bits; ``stream`` offsets the counter."""
    z = splitmix64(seed, np.arange(n, dtype=np.uint64) + np.uint64(stream) * np.uint64(1 << 40))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed, n, stream=0):
    """``n`` standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, n, stream=2 * stream + 1)
    u2 = uniform(seed, n, stream=2 * stream + 2)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
