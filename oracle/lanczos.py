"""Nested shift-invert Lanczos, Algorithm 1 (Sec. II), FP64.

Lanczos on (A - sigma I)^-1: each step solves (A - sigma) x = v_k (by the
MINRES of Algorithm 2, or a direct sparse solve when a test asks for speed),
then w = x - beta_k v_{k-1}; alpha_k = v_k . w; w -= alpha_k v_k. The basis is
orthonormalised against every previous vector (Fig. 1 caption: the new vector
is orthonormalised against the previous Lanczos basis vectors), here as a
second classical Gram-Schmidt pass. beta_{k+1} = ||w||; stop at beta_{k+1} = 0
or k = m. T_k (diagonal alpha, off-diagonal beta) is diagonalised and
(sigma + 1/theta_i, V_k y_i) returned.

Readings: the start vector is given by the caller; the wanted K pairs are the
K largest |theta| (eigenvalues nearest sigma), ordered by |E - sigma|.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import minres as _minres
from . import hamiltonian as _ham


def si_lanczos(solve, v, m, reorth=True):
    """Run Algorithm 1 for m steps. solve(v) -> (A - sigma)^-1 v.

    Returns (alpha[k], beta[k+1], V (n x k)): beta[0] = ||v||, beta[i] =
    beta_{i+1} for i >= 1.
    """
    n = len(v)
    V = np.zeros((n, m))
    alpha = np.zeros(m)
    beta = np.zeros(m + 1)
    beta[0] = np.linalg.norm(v)                 # beta_1
    v_prev = np.zeros(n)                        # v_0
    vk = v / beta[0]                            # v_1
    b_k = 0.0                                   # beta_k multiplying v_{k-1}; v_0 = 0
    k = 0
    while True:
        V[:, k] = vk
        x = solve(vk)                           # x = (A - sigma)^-1 v_k
        w = x - b_k * v_prev
        alpha[k] = vk @ w
        w = w - alpha[k] * vk
        if reorth:
            for _ in range(2):                  # full reorthogonalisation (CGS2)
                w = w - V[:, : k + 1] @ (V[:, : k + 1].T @ w)
        beta[k + 1] = np.linalg.norm(w)
        if beta[k + 1] == 0.0 or k + 1 == m:
            break
        v_prev, vk = vk, w / beta[k + 1]
        b_k = beta[k + 1]
        k += 1
    k += 1
    return alpha[:k], beta[: k + 1], V[:, :k]


def ritz(alpha, beta, V, sigma, K):
    """Diagonalise T_k; return the K pairs nearest sigma and SI residual
    estimates beta_{k+1} |y_{k,i}|."""
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[1:k], 1) + np.diag(beta[1:k], -1)
    theta, Y = np.linalg.eigh(T)
    order = np.argsort(-np.abs(theta), kind="stable")[:K]
    theta, Y = theta[order], Y[:, order]
    E = sigma + 1.0 / theta
    o2 = np.lexsort((E, np.abs(E - sigma)))
    theta, Y, E = theta[o2], Y[:, o2], E[o2]
    psi = V @ Y
    est = beta[k] * np.abs(Y[-1, :])
    return E, psi, theta, est


def sigma_midpoint(H, dense_limit=4000):
    """sigma = (E_min + E_max) / 2 (Sec. IV A)."""
    n = H.shape[0]
    if n <= dense_limit:
        w = np.linalg.eigvalsh(H.toarray())
        return 0.5 * (w[0] + w[-1])
    lo = sla.eigsh(H, k=1, which="SA", tol=1e-13, return_eigenvectors=False)[0]
    hi = sla.eigsh(H, k=1, which="LA", tol=1e-13, return_eigenvectors=False)[0]
    return 0.5 * (lo + hi)


def eigs_near(H, diag, sigma, K, v0, m, solver="minres", precond="row", tol=1e-12):
    """Full oracle pipeline: Algorithm 1 with Algorithm 2 inside."""
    n = H.shape[0]
    A = (H - sigma * sp.identity(n, format="csr")).tocsr()
    if solver == "minres":
        Minv = 1.0 / _ham.precond_diag(H, diag, sigma, precond)

        def solve(v):
            return _minres.pminres(A, v, Minv, tol=tol, kmax=50 * n)[0]
    else:
        lu = sla.splu(A.tocsc())

        def solve(v):
            return lu.solve(v)
    alpha, beta, V = si_lanczos(solve, v0, m)
    E, psi, theta, est = ritz(alpha, beta, V, sigma, K)
    res = np.array([np.linalg.norm(H @ psi[:, i] - E[i] * psi[:, i]) for i in range(psi.shape[1])])
    return E, psi, res
