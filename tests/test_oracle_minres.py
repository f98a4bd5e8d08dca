"""Oracle MINRES pins (Algorithm 2, Appendix A).

x_k must be the minimiser of ||b - A x||_{M^-1} over x_0 + K_k(M^-1 A, M^-1 r_0)
(Eq. (minres_solution) for the preconditioned system), computed here by brute
force: an explicit Krylov basis and a dense least-squares solve. |phi_k| must
equal that minimal residual norm, and the converged x must solve A x = b.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hamiltonian, minres
from paper_2203_09732_gb300 import inputs


def _system(L=8, h=3.0, seed=0, kind="row"):
    H, diag, st = hamiltonian.build(L, inputs.disorder(L, h, seed))
    sigma = 0.1234
    n = H.shape[0]
    A = (H - sigma * sp.identity(n)).toarray()
    M = hamiltonian.precond_diag(H, diag, sigma, kind)
    b = inputs.gaussian(n, 5)
    return A, M, b


@pytest.mark.parametrize("kind", ["id", "jacobi", "row"])
def test_dense_solve(kind):
    A, M, b = _system(kind=kind)
    x, k, phi = minres.pminres(A, b, 1.0 / M, tol=1e-13)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert k <= 4 * len(b)


@pytest.mark.parametrize("kind", ["id", "row"])
@pytest.mark.parametrize("x0seed", [None, 9])
def test_krylov_least_squares(kind, x0seed):
    A, M, b = _system(L=8, kind=kind)
    n = len(b)
    x0 = None if x0seed is None else inputs.gaussian(n, x0seed)
    xs_start = np.zeros(n) if x0 is None else x0
    x, k, phis, xs = minres.pminres(A, b, 1.0 / M, x0=x0, kmax=10, tol=0.0, history=True)
    Minv = 1.0 / M
    r0 = b - A @ xs_start
    W = np.sqrt(Minv)  # ||r||_{M^-1} = ||M^-1/2 r||
    K = [Minv * r0]
    for kk in range(1, 11):
        B = np.array(K).T
        # min_y || W (r0 - A B y) ||
        y, *_ = np.linalg.lstsq(W[:, None] * (A @ B), W * r0, rcond=None)
        xk = xs_start + B @ y
        assert np.linalg.norm(xs[kk] - xk) <= 1e-8 * max(1.0, np.linalg.norm(xk))
        res = np.linalg.norm(W * (b - A @ xs[kk]))
        assert abs(abs(phis[kk]) - res) <= 1e-9 * max(1.0, res)
        K.append(Minv * (A @ K[-1]))
        # re-orthonormalise the explicit basis columns for conditioning
        Q, _ = np.linalg.qr(np.array(K).T)
        K = list(Q.T)


def test_exact_in_n_steps():
    A, M, b = _system(L=8, kind="row")
    n = len(b)
    x, k, phi = minres.pminres(A, b, 1.0 / M, kmax=n, tol=0.0)
    assert np.linalg.norm(A @ x - b) <= 1e-6 * np.linalg.norm(b)


def test_zero_rhs_and_relative_stop():
    A, M, b = _system(L=6)
    x, k, phi = minres.pminres(A, np.zeros(len(b)), 1.0 / M)
    assert k == 0 and not x.any()
    x, k, phi = minres.pminres(A, b, 1.0 / M, tol=1e-6)
    beta1 = np.sqrt(b @ (b / M))
    assert abs(phi) < 1e-6 * beta1


def test_planted_sign_error_is_caught():
    """A mistake planted in a copy of the oracle (wrong sign of gamma_hat)
    must fail the brute-force Krylov pin."""
    import inspect
    src = inspect.getsource(minres.pminres)
    bad = src.replace("gamma_hat = -s_prev * delta_hat + c_prev * alpha",
                      "gamma_hat = s_prev * delta_hat + c_prev * alpha")
    assert bad != src
    ns = {"np": np}
    exec(bad, ns)
    A, M, b = _system(L=8)
    x, *_ = ns["pminres"](A, b, 1.0 / M, kmax=200, tol=1e-13)
    assert np.linalg.norm(A @ x - b) > 1e-6 * np.linalg.norm(b)
