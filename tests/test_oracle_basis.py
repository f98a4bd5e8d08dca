"""Oracle basis pins: brute force and closed-form counts (Sec. I: n = C(L, L/2))."""
import itertools
from math import comb

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16])
def test_dimension(L):
    assert len(basis.enumerate_states(L)) == comb(L, L // 2)


@pytest.mark.parametrize("L", [4, 6, 8, 10])
def test_against_itertools(L):
    ref = sorted(sum(1 << p for p in c) for c in itertools.combinations(range(L), L // 2))
    assert basis.enumerate_states(L).tolist() == ref


def test_rank_roundtrip():
    st = basis.enumerate_states(12)
    r = basis.rank(st, st)
    assert (r == np.arange(len(st))).all()
    assert basis.rank(st, np.array([0b111, 0b1111111]))[0] == -1


def test_chunked_enumeration_matches():
    a = basis.enumerate_states(14)
    b = basis.enumerate_states(14, chunk=1000)
    assert (a == b).all()


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12])
def test_counting_rank_matches_enumeration(L):
    st = basis.enumerate_states(L)
    for i in range(0, len(st), max(1, len(st) // 97)):
        assert basis.rank_count(st[i], L) == i
        assert basis.unrank_count(i, L) == st[i]
