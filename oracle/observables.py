"""The paper's other observables of the eigenpairs (Sec. IV B), FP64.

Bipartite entanglement entropy S = -Tr rho_A log rho_A (natural logarithm) of
a pure state psi for the subsystem A of sites j = 1..L/2 (bits 0..L/2-1): psi
is placed in the full 2^L space (index = state word), viewed as a
2^(L/2) x 2^(L/2) matrix (row = the bits of the other half, column = the bits
of A), and its squared singular values are the eigenvalues of rho_A. This
uses neither the Sz = 0 sector nor its rank order.

Level spacing ratio r_k = min(delta_k, delta_{k-1}) / max(delta_k, delta_{k-1})
with delta_k = E_{k+1} - E_k over the sorted eigenvalues.
"""
import numpy as np


def entanglement_entropy(psi, states, L):
    """S of the state(s) psi (vector of the sector in rank order, or an
    (n, K) array of columns); psi need not be normalised."""
    psi = np.asarray(psi, dtype=np.float64)
    cols = psi[:, None] if psi.ndim == 1 else psi
    half = L // 2
    out = []
    for c in cols.T:
        full = np.zeros(1 << L)
        full[np.asarray(states, dtype=np.int64)] = c / np.linalg.norm(c)
        sv = np.linalg.svd(full.reshape(1 << (L - half), 1 << half), compute_uv=False)
        lam = sv * sv
        lam = lam[lam > 0]
        out.append(float(-(lam * np.log(lam)).sum()))
    return out[0] if psi.ndim == 1 else np.array(out)


def level_spacing_ratios(E):
    """r_k for k = 2..K-1 (the K - 2 interior levels) of the eigenvalues E."""
    e = np.sort(np.asarray(E, dtype=np.float64))
    d = np.diff(e)
    lo = np.minimum(d[1:], d[:-1])
    hi = np.maximum(d[1:], d[:-1])
    return lo / hi


def s_rmt(L):
    """Random-matrix estimate of the entropy of the half chain (Sec. IV B)."""
    return np.log(2.0) / 2.0 * L + 0.5 * np.log(0.5) - 0.25
