"""torch.autograd interface to the eigenpairs' twist overlaps and energies.

TwistObservables.apply(h, L, K, sigma, seed, tol) returns, for the K
eigenpairs of H(h) nearest sigma (Eq. (1); nested shift-invert Lanczos with
MINRES, Algorithms 1 and 2), the squared twist overlaps |z_i|^2 (Sec. III) and
the energies E_i, as functions of the fields h (a float64 tensor of L
entries). The backward pass is the library's adjoint (hs_twist_grad): one
MINRES solve of (H - E_i) lambda = P (psi_i * u) per eigenpair for all L
derivatives of |z_i|^2, and Hellmann-Feynman dE_i/dh_j = -<Sz_j> for the
energies. Which eigenpairs are nearest sigma is held fixed (the selection is
piecewise constant in h); the eigenpairs must be non-degenerate.
"""
import numpy as np
import torch

from . import hs


class TwistObservables(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, L, K, sigma=float("nan"), seed=0, tol=1e-10):
        hv = h.detach().to(torch.float64).cpu().numpy()
        chain = hs.Chain(int(L), hv, sigma=float(sigma))
        ev, vecs, res, info = chain.eigs(int(K), seed=int(seed), minres_tol=min(tol, 1e-10))
        z = chain.twist(vecs)
        ctx.chain, ctx.vecs, ctx.ev, ctx.tol = chain, vecs, ev, tol
        ctx.h_device, ctx.h_dtype = h.device, h.dtype
        z2 = torch.from_numpy(np.abs(z) ** 2).to(h.dtype)
        E = torch.from_numpy(np.asarray(ev)).to(h.dtype)
        return z2.to(h.device), E.to(h.device)

    @staticmethod
    def backward(ctx, g_z2, g_E):
        z, dz2, dE, info = ctx.chain.twist_grad(ctx.vecs, ctx.ev, tol=ctx.tol)
        ctx.chain.close()
        gz = (g_z2.detach().to(torch.float64).cpu().numpy() if g_z2 is not None
              else np.zeros(dz2.shape[0]))
        gE = (g_E.detach().to(torch.float64).cpu().numpy() if g_E is not None
              else np.zeros(dE.shape[0]))
        grad = gz @ dz2 + gE @ dE
        return (torch.from_numpy(grad).to(ctx.h_dtype).to(ctx.h_device),
                None, None, None, None, None)


def twist_observables(h, L, K, sigma=float("nan"), seed=0, tol=1e-10):
    """(|z_i|^2, E_i) of the K eigenpairs nearest sigma, differentiable in h."""
    return TwistObservables.apply(h, L, K, sigma, seed, tol)
