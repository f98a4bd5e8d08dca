"""SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written from its published
definition, used as a counter-based generator: value i of stream ``seed`` is
mix(seed + (i + 1) * GAMMA). It draws the Lanczos start vector of Algorithm 1
(the paper leaves v unspecified); the library implements the same published
generator independently so both sides start from the same vector.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed, n):
    """n doubles in [-1, 1): 2 * (top 53 bits / 2^53) - 1."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GAMMA
        u = _mix(z) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0) * 2.0 - 1.0
