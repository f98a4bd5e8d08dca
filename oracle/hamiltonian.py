"""Explicit sparse Hamiltonian of Eq. (1) in the Sz = 0 sector, FP64.

H = sum_{j=1..L} ( S_j . S_{j+1} - h_j Sz_j ), periodic, J = 1.
S_j . S_{j+1} = Sz_j Sz_{j+1} + (S+_j S-_{j+1} + S-_j S+_{j+1}) / 2, so per bond:
  parallel pair      -> +1/4 on the diagonal,
  antiparallel pair  -> -1/4 on the diagonal and 1/2 between the state and the
                        state with both spins of the bond flipped (Appendix C:
                        the off-diagonal element is nonzero iff the two spins
                        are opposite).
The field adds -h_j * (+-1/2) on the diagonal.

Preconditioners of Sec. II (Eqs. for M_Jacobi and M_norm):
  Jacobi: diag |a_ii - sigma|;
  row norm: r_i = sqrt(|a_ii - sigma|^2 + sum_{k != i} |a_ik|^2);
  identity.
"""
import numpy as np
import scipy.sparse as sp

from . import basis


def bonds(L):
    """The L bonds (j, j+1 mod L), 0-based sites."""
    return [(j, (j + 1) % L) for j in range(L)]


def build(L, h, states=None):
    """Return (H as scipy CSR, diagonal, states)."""
    h = np.asarray(h, dtype=np.float64)
    if h.shape != (L,):
        raise ValueError("h must have L entries")
    if L < 4:
        raise ValueError("L >= 4 (at L = 2 the two bonds coincide)")
    if states is None:
        states = basis.enumerate_states(L)
    n = len(states)
    diag = np.zeros(n)
    rows, cols = [], []
    for (a, b) in bonds(L):
        sa = (states >> a) & 1
        sb = (states >> b) & 1
        anti = sa != sb
        diag += np.where(anti, -0.25, 0.25)
        idx = np.nonzero(anti)[0]
        tgt = basis.rank(states, states[idx] ^ ((1 << a) | (1 << b)))
        if (tgt < 0).any():
            raise AssertionError("bond flip left the Sz = 0 sector")
        rows.append(idx)
        cols.append(tgt)
    sz = basis.spins(states, L)
    diag -= sz @ h
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    off = sp.csr_matrix((np.full(len(r), 0.5), (r, c)), shape=(n, n))
    H = (off + sp.diags(diag)).tocsr()
    return H, diag, states


def dense(L, h):
    H, _, states = build(L, h)
    return H.toarray(), states


def precond_diag(H, diag, sigma, kind):
    """Diagonal of M for kind in {'id', 'jacobi', 'row'} (Sec. II)."""
    n = H.shape[0]
    if kind == "id":
        return np.ones(n)
    if kind == "jacobi":
        m = np.abs(diag - sigma)
        if (m == 0).any():
            raise ValueError("Jacobi preconditioner needs a_ii != sigma")
        return m
    if kind == "row":
        A = (H - sigma * sp.identity(n, format="csr")).tocsr()
        return np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    raise ValueError(kind)


def matvec(H, x, sigma=0.0):
    """(H - sigma) x with the explicit matrix."""
    return H @ x - sigma * x


def row(L, h, s, sigma=0.0):
    """Row of (H - sigma) for one state word s, from Eq. (1) directly:
    returns (diagonal a_ss - sigma, [(rank of flipped state, 1/2), ...]).
    Ranks come from basis.rank_count (no enumeration), for sampled rows at
    large L."""
    d = 0.0
    off = []
    for (a, b) in bonds(L):
        ba, bb = (s >> a) & 1, (s >> b) & 1
        if ba == bb:
            d += 0.25
        else:
            d -= 0.25
            off.append((basis.rank_count(s ^ ((1 << a) | (1 << b)), L), 0.5))
    for j in range(L):
        d -= h[j] * (0.5 if (s >> j) & 1 else -0.5)
    return d - sigma, off


def rownorm(L, h, s, sigma):
    """Row-norm preconditioner entry r_i of Sec. II for one state."""
    d, off = row(L, h, s, sigma)
    return np.sqrt(d * d + sum(v * v for _, v in off))
