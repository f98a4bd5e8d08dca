"""GPU parity of the observables of Sec. IV B: the entanglement entropy of
the library (reduced density blocks on the device, eigenvalues on the host)
against the oracle's full-space SVD, on eigenvectors from the eigensolver and
on random vectors; level spacing ratios of the library's eigenvalues."""
import numpy as np
import pytest

from oracle import basis, hamiltonian, observables as ob
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [4, 8, 12, 16])
def test_entropy_of_random_vectors(L):
    hs = need_gpu()
    st = basis.enumerate_states(L)
    V = inputs.gaussian(len(st), 40 + L, count=3)
    V[1] *= 7.5                       # not normalised: the call divides by the trace
    ref = ob.entanglement_entropy(V.T, st, L)
    with hs.Chain(L, inputs.disorder(L, 1.0, 0), sigma=0.0) as c:
        S = c.entanglement(to_dev(V))
    assert np.abs(S - ref).max() <= 1e-11 * max(1.0, ref.max())


def test_entropy_of_special_states():
    """A basis state: S = 0. Two basis states differing in both halves, weights
    p and 1 - p: S = -p ln p - (1-p) ln(1-p)."""
    hs = need_gpu()
    L = 10
    st = basis.enumerate_states(L)
    v = np.zeros((2, len(st)))
    v[0, basis.rank(st, 0b0011100101)] = 1.0
    p = 0.3
    v[1, basis.rank(st, 0b0000011111)] = np.sqrt(p)
    v[1, basis.rank(st, 0b1111100000)] = np.sqrt(1 - p)
    with hs.Chain(L, np.zeros(L), sigma=0.0) as c:
        S = c.entanglement(to_dev(v))
    assert abs(S[0]) < 1e-14
    assert abs(S[1] - (-p * np.log(p) - (1 - p) * np.log(1 - p))) < 1e-13


@pytest.mark.parametrize("L,h", [(12, 0.5), (14, 5.0)])
def test_entropy_and_level_ratio_of_eigenpairs(L, h):
    """Eigenpairs nearest sigma from the library: entropies against the
    oracle's on the same vectors and on dense eigh's vectors (eigenvectors are
    defined up to sign; the entropy is not affected), and the level ratios of
    the library's eigenvalues against the oracle's on dense eigenvalues."""
    hs = need_gpu()
    hv = inputs.disorder(L, h, 2)
    H, diag, st = hamiltonian.build(L, hv)
    w, Vd = np.linalg.eigh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    K = 12
    idx = np.lexsort((w, np.abs(w - sigma)))[:K]
    with hs.Chain(L, hv, sigma=sigma) as c:
        ev, vecs, res, info = c.eigs(K, seed=4)
        S = c.entanglement(vecs)
    assert np.abs(ev - w[idx]).max() < 1e-10
    ref = ob.entanglement_entropy(Vd[:, idx], st, L)
    assert np.abs(S - ref).max() <= 1e-9
    assert np.abs(S - ob.entanglement_entropy(vecs.cpu().numpy().T, st, L)).max() <= 1e-11
    r, mean = hs.level_ratio(ev)
    assert np.abs(r - ob.level_spacing_ratios(w[idx])).max() < 1e-6


def test_entropy_l20_eigenvector():
    """One eigenvector at L = 20 (the largest blocks are 252 x 252): against
    the oracle's SVD of the 1024 x 1024 full-space matrix."""
    hs = need_gpu()
    L = 20
    st = basis.enumerate_states(L)
    v = inputs.gaussian(len(st), 77, count=2)
    with hs.Chain(L, inputs.disorder(L, 3.0, 1), sigma=0.0) as c:
        S = c.entanglement(to_dev(v))
    ref = ob.entanglement_entropy(v.T, st, L)
    assert np.abs(S - ref).max() <= 1e-10 * ref.max()
