"""Oracle Hamiltonian pins (Eq. (1)).

The explicit sparse H is checked element by element against an independent
Kronecker-product construction in the full 2^L space, and against closed
forms and exact symmetries of Eq. (1).
"""
import os
from functools import reduce

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis, hamiltonian
from paper_2203_09732_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")

SX = np.array([[0, 0.5], [0.5, 0]])
SY = np.array([[0, -0.5j], [0.5j, 0]])
SZ = np.array([[0.5, 0], [0, -0.5]])  # basis index 0 = up (bit = 1 maps below)
I2 = np.eye(2)


def site_op(op, j, L):
    """op on site j (0-based) in the full space; full index bit j = 1 means up."""
    # numpy kron ordering: leftmost factor = most significant bit = site L-1.
    mats = [I2] * L
    mats[L - 1 - j] = op
    return reduce(np.kron, mats)


def full_H(L, h):
    # build with up = |1>: remap single-site ops to basis (|0>=down, |1>=up)
    P = np.array([[0, 1], [1, 0]])
    sx, sy, sz = (P @ m @ P for m in (SX, SY, SZ))
    H = np.zeros((1 << L, 1 << L), dtype=complex)
    for j in range(L):
        k = (j + 1) % L
        for op in (sx, sy, sz):
            H += site_op(op, j, L) @ site_op(op, k, L)
        H -= h[j] * site_op(sz, j, L)
    return H


@pytest.mark.parametrize("L", [4, 6, 8])
def test_matches_kronecker_construction(L):
    h = inputs.disorder(L, 2.0, 7)
    Hk = full_H(L, h)
    assert np.abs(Hk.imag).max() < 1e-14
    st = basis.enumerate_states(L)
    ref = Hk.real[np.ix_(st, st)]
    H, diag, _ = hamiltonian.build(L, h)
    assert np.abs(H.toarray() - ref).max() < 1e-13
    # the sector is closed: no matrix element leaves it ([H, Sz] = 0)
    out = np.setdiff1d(np.arange(1 << L), st)
    assert np.abs(Hk[np.ix_(out, st)]).max() < 1e-14


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14])
def test_trace_closed_form(L):
    # Tr H = -n L / (4 (L-1)) for any h: each bond is antiparallel with
    # probability L / (2 (L-1)) in the sector; the field traces to zero.
    h = inputs.disorder(L, 3.0, L)
    H, diag, st = hamiltonian.build(L, h)
    n = len(st)
    assert abs(diag.sum() - (-n * L / (4 * (L - 1)))) < 1e-9 * n


@pytest.mark.parametrize("L", [6, 8, 10])
def test_symmetric_and_offdiag_half(L):
    h = inputs.disorder(L, 1.0, 3)
    H, diag, st = hamiltonian.build(L, h)
    assert abs(H - H.T).max() == 0
    off = H - sp.diags(H.diagonal())
    off.eliminate_zeros()
    assert set(np.unique(off.data)) == {0.5}
    # row i has one off-diagonal per antiparallel bond
    nAF = sum(((st >> j) & 1) != ((st >> ((j + 1) % L)) & 1) for j in range(L))
    assert (np.diff(off.indptr) == nAF).all()


def _golden_spectra():
    rows = []
    for line in open(os.path.join(GOLD, "spectra.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append(line.split())
    return rows


def test_closed_form_spectra():
    for row in _golden_spectra():
        L = int(row[0])
        H, _ = hamiltonian.dense(L, np.zeros(L))
        w = np.linalg.eigvalsh(H)
        if row[2] == "min":
            assert abs(w[0] - float(row[3])) < 1e-12
        else:
            assert np.allclose(np.sort(w), sorted(map(float, row[2:])), atol=1e-12)


@pytest.mark.parametrize("L", [8, 10])
def test_spectral_symmetries(L):
    h = inputs.disorder(L, 3.0, 11)
    w = np.linalg.eigvalsh(hamiltonian.dense(L, h)[0])
    for hh in (-h, np.roll(h, 3), h[::-1]):
        w2 = np.linalg.eigvalsh(hamiltonian.dense(L, hh)[0])
        assert np.abs(w - w2).max() < 1e-11
    # a uniform field couples to Sz_tot = 0 only
    w0 = np.linalg.eigvalsh(hamiltonian.dense(L, np.zeros(L))[0])
    wu = np.linalg.eigvalsh(hamiltonian.dense(L, np.full(L, 1.7))[0])
    assert np.abs(w0 - wu).max() < 1e-11


@pytest.mark.parametrize("L", [6, 8])
def test_su2_multiplets(L):
    # at h = 0 every Sz = 1 eigenvalue is also an Sz = 0 eigenvalue
    Hk = full_H(L, np.zeros(L)).real
    full = np.arange(1 << L)
    pc = np.array([bin(s).count("1") for s in full])
    s1 = full[pc == L // 2 + 1]
    w1 = np.linalg.eigvalsh(Hk[np.ix_(s1, s1)])
    w0 = np.linalg.eigvalsh(hamiltonian.dense(L, np.zeros(L))[0])
    for e in w1:
        assert np.abs(w0 - e).min() < 1e-10


def test_preconditioners():
    L = 10
    h = inputs.disorder(L, 3.0, 0)
    H, diag, st = hamiltonian.build(L, h)
    sigma = 0.3
    D = H.toarray() - sigma * np.eye(H.shape[0])
    r = hamiltonian.precond_diag(H, diag, sigma, "row")
    assert np.allclose(r, np.linalg.norm(D, axis=1), rtol=1e-14)
    # every periodic Sz = 0 state has at least two antiparallel bonds
    assert r.min() >= np.sqrt(2) / 2 - 1e-15
    assert np.allclose(hamiltonian.precond_diag(H, diag, sigma, "jacobi"), np.abs(np.diag(D)))
    assert (hamiltonian.precond_diag(H, diag, sigma, "id") == 1).all()
    with pytest.raises(ValueError):
        hamiltonian.precond_diag(H, diag, diag[5], "jacobi")


@pytest.mark.parametrize("L", [6, 10])
def test_row_matches_explicit_matrix(L):
    h = inputs.disorder(L, 2.5, 4)
    H, diag, st = hamiltonian.build(L, h)
    D = H.toarray()
    sigma = 0.7
    for i in range(0, len(st), 7):
        d, off = hamiltonian.row(L, h, int(st[i]), sigma)
        ref = D[i].copy()
        ref[i] -= sigma
        mine = np.zeros(len(st))
        mine[i] = d
        for j, v in off:
            mine[j] += v
        assert np.abs(mine - ref).max() < 1e-13
        assert abs(hamiltonian.rownorm(L, h, int(st[i]), sigma) - np.linalg.norm(ref)) < 1e-12
