"""Oracle shift-invert Lanczos pins (Algorithm 1): the returned pairs are the
eigenpairs of H nearest sigma from a dense eigendecomposition."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hamiltonian, lanczos, rng
from paper_2203_09732_gb300 import inputs


@pytest.mark.parametrize("solver", ["direct", "minres"])
def test_matches_dense(solver):
    L = 10
    h = inputs.disorder(L, 3.0, 0)
    H, diag, st = hamiltonian.build(L, h)
    sigma = lanczos.sigma_midpoint(H)
    w = np.linalg.eigvalsh(H.toarray())
    K = 6
    v0 = rng.uniform_pm1(1, H.shape[0])
    E, psi, res = lanczos.eigs_near(H, diag, sigma, K, v0, m=60, solver=solver)
    ref = w[np.argsort(np.abs(w - sigma), kind="stable")[:K]]
    assert np.abs(np.sort(E) - np.sort(ref)).max() < 1e-10
    assert res.max() < 1e-8
    assert np.allclose(psi.T @ psi, np.eye(K), atol=1e-10)


def test_tridiagonal_projection():
    L = 8
    H, diag, st = hamiltonian.build(L, inputs.disorder(L, 2.0, 1))
    n = H.shape[0]
    sigma = 0.2
    Ainv = np.linalg.inv(H.toarray() - sigma * np.eye(n))
    a, b, V = lanczos.si_lanczos(lambda v: Ainv @ v, rng.uniform_pm1(3, n), 20)
    T = np.diag(a) + np.diag(b[1:len(a)], 1) + np.diag(b[1:len(a)], -1)
    assert np.allclose(V.T @ V, np.eye(len(a)), atol=1e-12)
    assert np.allclose(V.T @ Ainv @ V, T, atol=1e-10)


def test_sigma_midpoint():
    L = 12
    H, _, _ = hamiltonian.build(L, inputs.disorder(L, 3.0, 0))
    w = np.linalg.eigvalsh(H.toarray())
    assert abs(lanczos.sigma_midpoint(H, dense_limit=10) - 0.5 * (w[0] + w[-1])) < 1e-9


def test_golden_l12_matches_oracle():
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden", "l12_config.txt")
    rows = [l.split() for l in open(gold) if not l.startswith("#")]
    hv = np.array([float(x) for x in rows[0][1:]])
    assert np.array_equal(hv, inputs.disorder(12, 3.0, 0))
    sigma = float(rows[1][1])
    eigs = [float(r[1]) for r in rows if r[0] == "eig"]
    H, diag, st = hamiltonian.build(12, hv)
    E, psi, res = lanczos.eigs_near(H, diag, sigma, 10, rng.uniform_pm1(0, H.shape[0]), m=80,
                                    solver="minres")
    assert np.abs(np.sort(E) - np.sort(eigs)).max() < 1e-10
