"""Seeded synthetic inputs (no physics arithmetic lives here).

The paper's workloads are disorder realisations: h_j i.i.d. uniform on
[-h, h] (Sec. I, below Eq. (1)). Each realisation is drawn on the host with
numpy's PCG64 generator so both the CUDA path and the CPU oracle receive the
same FP64 array.
"""
import numpy as np


def disorder(L, h, seed):
    """h_1..h_L ~ U[-h, h] from seed."""
    return np.random.default_rng(seed).uniform(-h, h, L)


def disorder_mixed(L, seed, hlo=0.5, hhi=6.0):
    """Batched sweep recipe: h ~ U[hlo, hhi] per realisation, then h_j ~ U[-h, h]."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(hlo, hhi)
    return h, rng.uniform(-h, h, L)


def gaussian(n, seed, count=None):
    """N(0, 1) vector(s) in FP64 (shape (n,) or (count, n))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n if count is None else (count, n))


def dim(L):
    """C(L, L/2)."""
    from math import comb
    return comb(L, L // 2)


# The workloads the tests and the benchmark are built from.
WORKLOAD_L12 = dict(L=12, h=3.0, seeds=(0,), K=10, tol=1e-12)
WORKLOAD_L20 = dict(L=20, hs=(1.0, 2.0, 3.0, 4.0, 5.0), seeds=(0, 1, 2, 3, 4), K=20)
WORKLOAD_L28 = dict(L=28, h=3.7, seeds=(0, 1, 2), K=10)
