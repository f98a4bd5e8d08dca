"""Preconditioned MINRES, Algorithm 2 (Appendix A), FP64, written out step by
step in the paper's order and notation.

It solves A x = b for Hermitian (here real symmetric) A with a diagonal
positive definite preconditioner M = C C^T, i.e. MINRES on
(C^-1 A C^-T)(C^T x) = C^-1 b. Its iterate x_k minimises ||b - A x||_{M^-1}
over x_0 + K_k(M^-1 A, M^-1 r_0) (Eq. (minres_solution), preconditioned), and
|phi_k| equals that minimal residual norm.

Readings where the listing is silent:
  * epsilon_1 is read before it is set; it multiplies d_{-1} = 0, so it is 0;
  * the stopping test compares |phi_k| with tol * beta_1 (relative) instead of
    the absolute tol of the listing;
  * a zero beta_{k+1} (exact invariant subspace) ends the loop after the update.
"""
import numpy as np


def pminres(A, b, Minv, x0=None, kmax=None, tol=1e-12, history=False):
    """A: callable x -> A x (or a matrix); Minv: diagonal of M^-1 (array).

    Returns (x, k, phi_k) or, with history=True, (x, k, phis, xs) where xs[k]
    is x_k (k = 0..) for brute-force checks on tiny problems.
    """
    mv = A if callable(A) else (lambda v: A @ v)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if kmax is None:
        kmax = 10 * n
    # initialisation
    z_prev = np.zeros(n)                      # z_0
    z = b - mv(x)                             # z_1
    q = Minv * z                              # q_1
    beta_prev = 1.0                           # beta_0
    beta = np.sqrt(q @ z)                     # beta_1
    beta1 = beta
    phi = beta                                # phi_0
    delta_hat = 0.0                           # hat delta_1
    c_prev, s_prev = 1.0, 0.0                 # c_0, s_0
    eps = 0.0                                 # epsilon_1 (reading)
    d_prev2 = np.zeros(n)                     # d_{-1}
    d_prev = np.zeros(n)                      # d_0
    k = 0
    phis, xs = [phi], [x.copy()]
    if beta == 0.0:
        return (x, 0, phis, xs) if history else (x, 0, 0.0)
    while abs(phi) >= tol * beta1 and k < kmax:
        k += 1
        p = mv(q)                                             # p_k = A q_k
        alpha = (q @ p) / beta ** 2                           # alpha_k
        z_next = p / beta - (alpha / beta) * z - (beta / beta_prev) * z_prev
        q_next = Minv * z_next                                # q_{k+1}
        beta_next = np.sqrt(max(q_next @ z_next, 0.0))        # beta_{k+1}
        delta = c_prev * delta_hat + s_prev * alpha           # delta_k
        gamma_hat = -s_prev * delta_hat + c_prev * alpha      # hat gamma_k
        eps_next = s_prev * beta_next                         # epsilon_{k+1}
        delta_hat_next = c_prev * beta_next                   # hat delta_{k+1}
        gamma = np.sqrt(gamma_hat ** 2 + beta_next ** 2)      # gamma_k
        c = gamma_hat / gamma                                 # c_k
        s = beta_next / gamma                                 # s_k
        tau = c * phi                                         # tau_k
        phi = -s * phi                                        # phi_k
        d = (q / beta - delta * d_prev - eps * d_prev2) / gamma   # d_k
        x = x + tau * d                                       # x_k
        # shift k -> k + 1
        z_prev, z = z, z_next
        q = q_next
        beta_prev, beta = beta, beta_next
        delta_hat, eps = delta_hat_next, eps_next
        c_prev, s_prev = c, s
        d_prev2, d_prev = d_prev, d
        if history:
            phis.append(phi)
            xs.append(x.copy())
        if beta_next == 0.0:
            break
    return (x, k, phis, xs) if history else (x, k, phi)
