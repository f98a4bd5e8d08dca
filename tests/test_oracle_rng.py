"""SplitMix64 against its published test vector (seed 1234567)."""
import os

import numpy as np

from oracle import rng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_published_vector():
    ref = [int(l) for l in open(os.path.join(GOLD, "splitmix64.txt")) if not l.startswith("#")]
    with np.errstate(over="ignore"):
        z = np.uint64(1234567) + np.arange(1, 6, dtype=np.uint64) * rng.GAMMA
        out = rng._mix(z)
    assert [int(v) for v in out] == ref


def test_uniform_range():
    u = rng.uniform_pm1(7, 100000)
    assert u.min() >= -1 and u.max() < 1
    assert abs(u.mean()) < 0.01
