"""GPU parity of the adjoint derivatives of the eigenpairs' twist overlaps
(hs_twist_grad, and the torch.autograd.Function behind it) against the
oracle: central finite differences (step 1e-5, FP64) of |z|^2 and E from the
oracle's dense eigenpairs and direct twist sum, Hellmann-Feynman
dE/dh_j = -<Sz_j> from the oracle's spins, and two exact sum rules (a uniform
field couples to Sz_tot = 0, so it changes neither E nor psi)."""
import numpy as np
import pytest

from oracle import basis, hamiltonian, twist
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, torch

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _dense_pairs(L, h, sigma, K):
    """The K eigenpairs nearest sigma by dense eigh, ordered by |E - sigma|."""
    H, diag, st = hamiltonian.build(L, h)
    w, V = np.linalg.eigh(H.toarray())
    idx = np.lexsort((w, np.abs(w - sigma)))[:K]
    return w[idx], V[:, idx], st


def _fd(L, h, sigma, K):
    """Central differences of |z_i|^2 and E_i with respect to every h_j."""
    dz2 = np.zeros((K, L))
    dE = np.zeros((K, L))
    for j in range(L):
        out = []
        for sgn in (1, -1):
            hh = h.copy()
            hh[j] += sgn * EPS
            E, V, st = _dense_pairs(L, hh, sigma, K)
            out.append((E, np.abs(twist.overlap(V, st, L)) ** 2))
        dE[:, j] = (out[0][0] - out[1][0]) / (2 * EPS)
        dz2[:, j] = (out[0][1] - out[1][1]) / (2 * EPS)
    return dz2, dE


@pytest.mark.parametrize("L,hh,seed", [(8, 3.0, 1), (10, 2.0, 3), (12, 4.0, 5)])
def test_adjoint_matches_finite_differences_and_hellmann_feynman(L, hh, seed):
    hs = need_gpu()
    h = inputs.disorder(L, hh, seed)
    H, diag, st = hamiltonian.build(L, h)
    w = np.linalg.eigvalsh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    K = 4
    E0, V0, _ = _dense_pairs(L, h, sigma, K)
    gaps = np.min(np.abs(E0[:, None] - w[None, :]) + np.where(np.isclose(E0[:, None], w[None, :]), 1e9, 0), axis=1)
    assert gaps.min() > 1e-3, "nearly degenerate pair: finite differences would not resolve it"
    with hs.Chain(L, h, sigma=sigma) as c:
        ev, vecs, res, info = c.eigs(K, seed=7)
        z, dz2, dE, ginfo = c.twist_grad(vecs, ev)
        assert abs(c.sigma - sigma) < 1e-15          # restored
    assert np.abs(ev - E0).max() < 1e-10
    # Hellmann-Feynman against the oracle's <Sz_j>: dE/dh_j = -sum psi^2 s_j
    sz = basis.spins(st, L)
    hf = -(V0 ** 2).T @ sz
    assert np.abs(dE - hf).max() < 1e-11
    # against central differences of the oracle's dense eigenpairs
    fd_z2, fd_E = _fd(L, h, sigma, K)
    assert np.abs(dE - fd_E).max() < 1e-7
    scale = max(1.0, np.abs(fd_z2).max())
    assert np.abs(dz2 - fd_z2).max() <= 1e-6 * scale, (dz2, fd_z2)
    # |z| itself against the oracle's direct sum
    assert np.abs(np.abs(z) ** 2 - np.abs(twist.overlap(V0, st, L)) ** 2).max() < 1e-11
    # sum rules of a uniform field
    assert np.abs(dE.sum(axis=1)).max() < 1e-12
    assert np.abs(dz2.sum(axis=1)).max() < 1e-8 * scale


def test_autograd_function_gives_the_adjoint():
    """The torch.autograd.Function: backward of a weighted sum of |z_i|^2 and
    E_i equals the same combination of the adjoint rows, and a directional
    finite difference of the forward agrees."""
    need_gpu()
    from paper_2203_09732_gb300 import autograd as ag, hs
    L, K = 10, 3
    h0 = inputs.disorder(L, 2.5, 11)
    H, diag, st = hamiltonian.build(L, h0)
    w = np.linalg.eigvalsh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    a = torch.tensor([0.3, -1.0, 0.7], dtype=torch.float64)
    b = torch.tensor([0.1, 0.2, -0.4], dtype=torch.float64)
    h = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    z2, E = ag.twist_observables(h, L, K, sigma=sigma, seed=3)
    loss = (a * z2).sum() + (b * E).sum()
    loss.backward()
    g = h.grad.numpy()
    # directional finite difference of the forward along a random direction
    d = np.random.default_rng(2).standard_normal(L)
    vals = []
    for sgn in (1, -1):
        hp = torch.tensor(h0 + sgn * EPS * d, dtype=torch.float64)
        z2p, Ep = ag.twist_observables(hp, L, K, sigma=sigma, seed=3)
        vals.append(float((a * z2p).sum() + (b * Ep).sum()))
    fd = (vals[0] - vals[1]) / (2 * EPS)
    assert abs(g @ d - fd) <= 1e-6 * max(1.0, abs(fd)), (g @ d, fd)
