"""Oracle twist pins (Sec. III, Appendix B): hand-computed u_alpha, |z| <= 1,
the Lemma sum_alpha u_alpha = 0, z -> -z under translation, and the thermal
Gaussian estimate E|z|^2 = 2/n (Eq. (twist_thermal_gaussian))."""
import os

import numpy as np
import pytest

from oracle import basis, hamiltonian, twist
from paper_2203_09732_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_computed_states():
    for line in open(os.path.join(GOLD, "twist_states.txt")):
        if line.startswith("#") or not line.strip():
            continue
        L, s, re, im = line.split()
        u = twist.u_diag(np.array([int(s)]), int(L))[0]
        assert abs(u - complex(float(re), float(im))) < 1e-14


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16])
def test_lemma_sum_u_zero(L):
    u = twist.u_diag(basis.enumerate_states(L), L)
    assert abs(u.sum()) < 1e-9
    assert np.allclose(np.abs(u), 1.0)


def test_bounds_and_basis_state():
    L = 10
    st = basis.enumerate_states(L)
    psi = inputs.gaussian(len(st), 1)
    psi /= np.linalg.norm(psi)
    assert abs(twist.overlap(psi, st, L)) <= 1.0
    e = np.zeros(len(st))
    e[17] = 1.0
    assert abs(abs(twist.overlap(e, st, L)) - 1.0) < 1e-14


def test_translation_flips_sign():
    # T^dagger U T = -U (Appendix B): eigenstates of the translated disorder
    # have the opposite z.
    L = 10
    h = inputs.disorder(L, 3.0, 2)
    st = basis.enumerate_states(L)
    w1, V1 = np.linalg.eigh(hamiltonian.dense(L, h)[0])
    w2, V2 = np.linalg.eigh(hamiltonian.dense(L, np.roll(h, 1))[0])
    assert np.abs(w1 - w2).max() < 1e-10
    gaps = np.diff(w1)
    pick = [i for i in range(1, len(w1) - 1) if min(gaps[i - 1], gaps[i]) > 1e-6][:20]
    z1 = twist.overlap(V1[:, pick], st, L)
    z2 = twist.overlap(V2[:, pick], st, L)
    assert np.abs(z1 + z2).max() < 1e-9


def test_gaussian_mean_two_over_n():
    L = 8
    st = basis.enumerate_states(L)
    n = len(st)
    c = inputs.gaussian(n, 123, count=20000) / np.sqrt(n)
    z = twist.overlap(c.T, st, L)
    z2 = np.abs(z) ** 2
    mean, se = z2.mean(), z2.std() / np.sqrt(len(z2))
    assert abs(mean - 2.0 / n) < 4 * se


def test_u_is_unitary_diagonal_of_full_space_operator():
    # build exp(i 2pi/L sum_j j Sz_j) in the full space by brute force
    L = 6
    full = np.arange(1 << L)
    phase = np.zeros(len(full))
    for j in range(1, L + 1):
        phase += j * np.where((full >> (j - 1)) & 1, 0.5, -0.5)
    U = np.exp(1j * 2 * np.pi / L * phase)
    st = basis.enumerate_states(L)
    assert np.allclose(twist.u_diag(st, L), U[st], atol=1e-15)
