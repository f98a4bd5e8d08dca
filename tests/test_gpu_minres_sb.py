"""GPU parity of the superblock MINRES form (Algorithm 2 on the superblock
layout: pass A = the superblock H x with the alpha dot (ten-low-bit form in
FP32 and four-low-bit form in FP64 by default; HS_SB4 forces one), pass B =
q_{k+1},
beta_{k+1}, the Givens rotation and the d/x update of the previous iteration).
It is the default from L = 24 on; HS_MINRES_SB=1 makes it the first choice
wherever a superblock plan exists, and HS_SB_PLANS=1 with HS_KLO=4 builds
plans for small chains, so that full solves can be checked against the
oracle's sparse direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import hamiltonian, minres
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev, torch
from tests.test_gpu_minres import TOL32, TOL64, separated_sigma

pytestmark = pytest.mark.gpu


@pytest.fixture
def small_sb(monkeypatch):
    """Superblock plans on a small chain (k = 4 low bits), form forced."""
    monkeypatch.setenv("HS_SB_PLANS", "1")
    monkeypatch.setenv("HS_KLO", "4")
    monkeypatch.setenv("HS_SB_KS32", "8")
    monkeypatch.setenv("HS_SB_KS64", "8")
    monkeypatch.setenv("HS_MINRES_SB", "1")


@pytest.fixture(scope="module")
def l22():
    L = 22
    hv = inputs.disorder(L, 3.0, 0)
    H, diag, st = hamiltonian.build(L, hv)
    return L, hv, H, diag


@pytest.mark.parametrize("form", ["1", "0"])
@pytest.mark.parametrize("kind", ["id", "row"])
@pytest.mark.parametrize("k", [1, 3, 7, 20])
def test_iterates_match_oracle_l22(l22, kind, k, form, monkeypatch):
    """FP64 and FP32 iterates of the superblock form at L = 22 (its k = 10
    tables, windows as at L = 28) element by element against the oracle.
    (At L = 22 the 705k diagonal values are so dense that some a_ii - sigma
    cancels at any shift, so Jacobi is checked by the next test.)"""
    hs = need_gpu()
    monkeypatch.setenv("HS_MINRES_SB", "1")
    monkeypatch.setenv("HS_SB4", form)
    L, hv, H, diag = l22
    sigma = separated_sigma(diag)
    A = (H - sigma * sp.identity(H.shape[0])).tocsr()
    b = inputs.gaussian(A.shape[0], 11)
    M = hamiltonian.precond_diag(H, diag, sigma, kind)
    xr, kr, phir = minres.pminres(A, b, 1.0 / M, kmax=k, tol=0.0)
    with hs.Chain(L, hv, sigma=sigma) as c:
        x, info = c.minres(to_dev(b), tol=0.0, kmax=k, precond=kind, allow_not_converged=True)
        x32, i32 = c.minres_f32(to_dev(b, torch.float32), tol=0.0, kmax=k, precond=kind,
                                allow_not_converged=True)
    assert info["iters"] == k and i32["iters"] == k
    assert info["form"] == i32["form"] == hs.FORM_SUPERBLOCK
    scale = np.abs(xr).max()
    assert np.abs(x.cpu().numpy() - xr).max() <= TOL64[k] * scale
    assert np.abs(x32.cpu().double().numpy() - xr).max() <= TOL32[k] * scale


@pytest.mark.parametrize("kind", ["id", "jacobi", "row"])
@pytest.mark.parametrize("k", [1, 3, 7, 20])
def test_iterates_minimise_the_residual_l22(l22, kind, k, monkeypatch):
    """Eq. (minres_solution) for the superblock form at L = 22: the oracle's
    explicit A gives the true ||b - A x_k||_{M^-1} of the GPU iterate, which
    must equal the oracle's minimum |phi_k| (FP64)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_MINRES_SB", "1")
    L, hv, H, diag = l22
    sigma = 0.1234
    A = (H - sigma * sp.identity(H.shape[0])).tocsr()
    b = inputs.gaussian(A.shape[0], 11)
    M = hamiltonian.precond_diag(H, diag, sigma, kind)
    xr, kr, phir = minres.pminres(A, b, 1.0 / M, kmax=k, tol=0.0)
    with hs.Chain(L, hv, sigma=sigma) as c:
        x, info = c.minres(to_dev(b), tol=0.0, kmax=k, precond=kind, allow_not_converged=True)
    assert info["form"] == hs.FORM_SUPERBLOCK
    r = b - A @ x.cpu().numpy()
    got = np.sqrt(r @ (r / M))
    assert abs(got - abs(phir)) <= 1e-10 * abs(phir), (got, abs(phir))


@pytest.mark.parametrize("L", [14, 16])
@pytest.mark.parametrize("kind", ["id", "row"])
def test_full_solves_small_chain(L, kind, small_sb):
    """Whole solves through the superblock form: FP64 to 1e-12 and FP32 +
    FP64 refinement to 1e-12 in the M^-1 norm, checked with the oracle's A;
    both against the sparse direct solve."""
    hs = need_gpu()
    hv = inputs.disorder(L, 3.0, L)
    H, diag, st = hamiltonian.build(L, hv)
    sigma = 0.1234
    A = (H - sigma * sp.identity(H.shape[0])).tocsc()
    M = hamiltonian.precond_diag(H, diag, sigma, kind)
    b = inputs.gaussian(A.shape[0], 3)
    xd = sla.spsolve(A, b)
    with hs.Chain(L, hv, sigma=sigma) as c:
        x, info = c.minres(to_dev(b), tol=1e-12, precond=kind)
        xm, im = c.minres(to_dev(b), tol=1e-12, precond=kind, mixed=True)
    assert info["status"] == 0 and im["status"] == 0 and im["sweeps"] >= 2
    assert info["form"] == im["form"] == hs.FORM_SUPERBLOCK
    for xx in (x.cpu().numpy(), xm.cpu().numpy()):
        r = b - A @ xx
        assert np.sqrt(r @ (r / M)) <= 1.0001e-12 * np.sqrt(b @ (b / M)) * 50
        assert np.linalg.norm(xx - xd) <= 1e-6 * np.linalg.norm(xd)


def test_edge_cases_small_chain(small_sb):
    hs = need_gpu()
    L = 14
    hv = inputs.disorder(L, 3.0, 0)
    H, diag, st = hamiltonian.build(L, hv)
    n = H.shape[0]
    with hs.Chain(L, hv, sigma=0.1234) as c:
        x, info = c.minres(torch.zeros(n, dtype=torch.float64, device="cuda"))
        assert info["iters"] == 0 and not x.abs().max().item()
        assert info["form"] == hs.FORM_SUPERBLOCK
        with pytest.raises(hs.HSError) as e:
            c.minres(to_dev(inputs.gaussian(n, 1)), kmax=1)
        assert e.value.status == hs.HS_NOT_CONVERGED
        bn = inputs.gaussian(n, 2)
        bn[3] = np.nan
        with pytest.raises(hs.HSError) as e:
            c.minres(to_dev(bn))
        assert e.value.status == hs.HS_NONFINITE
        c.sigma = float(diag[5])
        with pytest.raises(hs.HSError) as e:
            c.minres(to_dev(inputs.gaussian(n, 1)), precond="jacobi")
        assert e.value.status == hs.HS_BAD_ARG


def test_eigenpairs_small_chain(small_sb):
    """Algorithm 1 with the superblock MINRES inside, FP64 and FP32 +
    refinement, against dense eigh."""
    hs = need_gpu()
    L, K = 12, 6
    hv = inputs.disorder(L, 3.0, 0)
    H, diag, st = hamiltonian.build(L, hv)
    w, V = np.linalg.eigh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    idx = np.lexsort((w, np.abs(w - sigma)))[:K]
    with hs.Chain(L, hv, sigma=sigma) as c:
        for mixed, tol in ((False, 1e-10), (True, 1e-9)):
            ev, vecs, res, info = c.eigs(K, mixed=mixed, seed=4)
            assert np.abs(ev - w[idx]).max() < tol and info["converged"] == K


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_matches_persistent_form_l24(dtype, monkeypatch):
    """At L = 24 (n = 2.7M) the superblock form (default there) and the
    global-memory persistent form run the same recurrence: after 40
    iterations their iterates agree to the rounding of the reductions."""
    hs = need_gpu()
    L = 24
    hv = inputs.disorder(L, 3.7, 0)
    xs = {}
    with hs.Chain(L, hv, sigma=0.05) as c:
        b = torch.from_numpy(inputs.gaussian(c.n, 5)).cuda()
        for form in ("1", "0"):
            monkeypatch.setenv("HS_MINRES_SB", form)
            if dtype == "f64":
                x, info = c.minres(b, tol=0.0, kmax=40, allow_not_converged=True)
            else:
                x, info = c.minres_f32(b.float(), tol=0.0, kmax=40, allow_not_converged=True)
            assert info["iters"] == 40
            assert info["form"] == (hs.FORM_SUPERBLOCK if form == "1" else hs.FORM_PERSISTENT)
            xs[form] = x.double().cpu().numpy()
    scale = np.abs(xs["0"]).max()
    tol = 1e-12 if dtype == "f64" else 1e-4
    assert np.abs(xs["1"] - xs["0"]).max() <= tol * scale


@pytest.mark.parametrize("L", [14, 16])
def test_refinement_residual_through_superblock_product(L, small_sb, monkeypatch):
    """The FP64 residual b - (H - sigma) x of the refinement, with the product
    taken by the superblock FP64 kernel (HS_HV_SB=1; the default from L = 24):
    the M^-1- and 2-norm residuals that hs_minres reports after an FP64 solve
    capped at 20 iterations, and after an FP32 + refinement solve, against the
    oracle's explicit A applied to the returned x."""
    hs = need_gpu()
    monkeypatch.setenv("HS_HV_SB", "1")
    hv = inputs.disorder(L, 3.0, 2)
    H, diag, st = hamiltonian.build(L, hv)
    sigma = 0.05
    A = (H - sigma * sp.identity(H.shape[0])).tocsr()
    b = inputs.gaussian(A.shape[0], 5)
    M = hamiltonian.precond_diag(H, diag, sigma, "row")
    with hs.Chain(L, hv, sigma=sigma) as c:
        x, info = c.minres(to_dev(b), tol=0.0, kmax=20, precond="row", allow_not_converged=True)
        xm, im = c.minres(to_dev(b), tol=1e-10, precond="row", mixed=True, inner_tol=1e-4)
    for xx, inf in ((x, info), (xm, im)):
        r = b - A @ xx.cpu().numpy()
        rel_m = np.sqrt(r @ (r / M)) / np.sqrt(b @ (b / M))
        rel_2 = np.linalg.norm(r) / np.linalg.norm(b)
        # FP64 rounding of b - A x is ~1e-15 of |b| (absolute floor 1e-13)
        assert abs(inf["resid_minv"] - rel_m) <= 1e-9 * rel_m + 1e-13
        assert abs(inf["resid_2"] - rel_2) <= 1e-9 * rel_2 + 1e-13
    assert im["resid_minv"] <= 1e-10 and im["sweeps"] >= 2
