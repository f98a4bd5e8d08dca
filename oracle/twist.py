"""Twist overlap z = <psi| U_twist |psi>, U_twist = exp[i 2pi/L sum_j j Sz_j]
(Sec. III), by the direct sum z = sum_alpha c_alpha^2 u_alpha with
u_alpha = <alpha|U_twist|alpha> (Appendix B), in complex128.
"""
import numpy as np

from . import basis


def u_diag(states, L):
    """u_alpha for every basis state: exp(i 2pi/L sum_{j=1..L} j Sz_j)."""
    sz = basis.spins(states, L)                       # (n, L), site j at column j-1
    phase = sz @ np.arange(1, L + 1, dtype=np.float64)
    return np.exp(1j * 2.0 * np.pi / L * phase)


def overlap(psi, states, L):
    """z for real psi (vector or (n, K) matrix of columns)."""
    u = u_diag(states, L)
    c2 = np.asarray(psi, dtype=np.float64) ** 2
    if c2.ndim == 1:
        return np.sum(c2 * u)
    return (u[:, None] * c2).sum(axis=0)
