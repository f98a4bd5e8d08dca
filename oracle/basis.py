"""Sz = 0 sector basis by brute force (Sec. I below Eq. (1): even L, Sz = 0,
dimension n = C(L, L/2)).

A state is an L-bit word; bit j-1 holds site j, bit = 1 is spin up. The sector
is every word with popcount L/2, in ascending integer order; the rank of a
state is its position in that list (found by binary search, no combinatorics).
"""
import numpy as np


def _popcount(a):
    a = a.astype(np.uint64, copy=True)
    c = np.zeros(a.shape, dtype=np.int64)
    while True:
        nz = a != 0
        if not nz.any():
            return c
        c += nz
        a &= a - np.uint64(1)  # clear lowest set bit


def enumerate_states(L, chunk=1 << 24):
    """All L-bit words with popcount L/2, ascending (int64)."""
    if L % 2 or L < 2:
        raise ValueError("L must be even and >= 2")
    out = []
    for lo in range(0, 1 << L, chunk):
        a = np.arange(lo, min(lo + chunk, 1 << L), dtype=np.int64)
        out.append(a[_popcount(a) == L // 2])
    return np.concatenate(out)


def rank(states, s):
    """Rank of state word(s) s in the ascending list ``states``; -1 if absent."""
    s = np.asarray(s, dtype=np.int64)
    r = np.searchsorted(states, s)
    r = np.minimum(r, len(states) - 1)
    return np.where(states[r] == s, r, -1)


def spins(states, L):
    """Sz_j of each state as an (n, L) float array of +-1/2, column j-1 = site j."""
    bits = (states[:, None] >> np.arange(L)[None, :]) & 1
    return np.where(bits == 1, 0.5, -0.5)


def _binom(n, r):
    from math import comb
    return comb(n, r) if 0 <= r <= n else 0


def rank_count(s, L):
    """Rank of one state word by counting the sector words below it: for every
    set bit p (scanned from the top), the words that agree above p and have 0
    at p number C(p, remaining ones). No table; used for large L."""
    s = int(s)
    ones = L // 2
    r = 0
    for p in range(L - 1, -1, -1):
        if (s >> p) & 1:
            r += _binom(p, ones)
            ones -= 1
    return r


def unrank_count(r, L):
    """Inverse of rank_count: the state word of rank r."""
    r = int(r)
    ones = L // 2
    s = 0
    for p in range(L - 1, -1, -1):
        if ones == 0:
            break
        c = _binom(p, ones)
        if r >= c:
            s |= 1 << p
            r -= c
            ones -= 1
    return s
