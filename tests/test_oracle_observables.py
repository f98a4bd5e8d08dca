"""Pins of the oracle's observables (Sec. IV B): entanglement entropy
against closed forms of product, singlet and Bell states and against the
paper's random-matrix value; level spacing ratio against exact small cases
and the Poisson and GOE values the paper quotes."""
import numpy as np
import pytest

from oracle import basis, observables as ob
from paper_2203_09732_gb300 import inputs


def _state(L, amps):
    """Sector vector with the given {state word: amplitude}."""
    st = basis.enumerate_states(L)
    v = np.zeros(len(st))
    for s, a in amps.items():
        v[basis.rank(st, s)] = a
    return v, st


def test_basis_state_has_no_entanglement():
    L = 8
    v, st = _state(L, {0b00110110: 1.0})
    assert abs(ob.entanglement_entropy(v, st, L)) < 1e-14


def test_singlets_inside_and_across_the_cut():
    """L = 4, A = sites 1, 2. Singlets on bonds (1,2) and (3,4) lie inside the
    halves: S = 0. Singlets on (2,3) and (4,1) both cross the cut: S = 2 ln 2.
    (Site j is bit j-1.)"""
    L = 4

    def singlet_pair(p, q):
        # (|up_p down_q> - |down_p up_q>) / sqrt(2) on two sites, as {bits: amp}
        return {(1 << p): 1 / np.sqrt(2), (1 << q): -1 / np.sqrt(2)}

    def product(d1, d2):
        out = {}
        for s1, a1 in d1.items():
            for s2, a2 in d2.items():
                out[s1 | s2] = out.get(s1 | s2, 0.0) + a1 * a2
        return out

    v, st = _state(L, product(singlet_pair(0, 1), singlet_pair(2, 3)))
    assert abs(ob.entanglement_entropy(v, st, L)) < 1e-14
    v, st = _state(L, product(singlet_pair(1, 2), singlet_pair(3, 0)))
    assert abs(ob.entanglement_entropy(v, st, L) - 2 * np.log(2)) < 1e-14


def test_equal_superposition_across_the_cut():
    """Two basis states that differ in both halves, weights p and 1 - p:
    S = -p ln p - (1-p) ln(1-p)."""
    L = 6
    p = 0.3
    v, st = _state(L, {0b000111: np.sqrt(p), 0b111000: np.sqrt(1 - p)})
    ref = -p * np.log(p) - (1 - p) * np.log(1 - p)
    assert abs(ob.entanglement_entropy(v, st, L) - ref) < 1e-14


def test_entropy_of_random_sector_states_approaches_the_rmt_value():
    """Gaussian random vectors of the Sz = 0 sector: their mean entropy
    approaches S_RMT(L) of the paper (measured: 0.042 below at L = 8, 0.005 at
    L = 14)."""
    L = 14
    st = basis.enumerate_states(L)
    vals = [ob.entanglement_entropy(inputs.gaussian(len(st), s), st, L) for s in range(20)]
    assert abs(np.mean(vals) - ob.s_rmt(L)) < 0.02
    # and it never exceeds the largest possible value, ln of the smaller dimension
    assert max(vals) < (L // 2) * np.log(2)


def test_entropy_is_symmetric_under_the_cut_and_sign():
    L = 10
    st = basis.enumerate_states(L)
    v = inputs.gaussian(len(st), 3)
    assert abs(ob.entanglement_entropy(v, st, L) - ob.entanglement_entropy(-2.5 * v, st, L)) < 1e-12


def test_level_ratio_small_cases():
    assert np.allclose(ob.level_spacing_ratios([0.0, 1.0, 3.0]), [0.5])
    assert np.allclose(ob.level_spacing_ratios([3.0, 0.0, 1.0, 6.0]), [0.5, 2.0 / 3.0])
    assert np.allclose(ob.level_spacing_ratios(np.arange(7.0)), 1.0)


def test_level_ratio_poisson_and_goe():
    """Uncorrelated levels (exponential spacings): mean r = 2 ln 2 - 1; levels
    from the middle of GOE matrices: mean r = 0.5307 (values quoted in Sec. IV B),
    each within four standard errors of the sample."""
    rng = np.random.default_rng(0)
    rp = np.concatenate([ob.level_spacing_ratios(np.cumsum(rng.exponential(size=2000)))
                         for _ in range(50)])
    assert abs(rp.mean() - (2 * np.log(2) - 1)) < 4 * rp.std() / np.sqrt(len(rp))
    rg = []
    for _ in range(100):
        A = rng.standard_normal((300, 300))
        w = np.linalg.eigvalsh((A + A.T) / 2)
        rg.append(ob.level_spacing_ratios(w[100:200]))
    rg = np.concatenate(rg)
    assert abs(rg.mean() - 0.5307) < 4 * rg.std() / np.sqrt(len(rg))
