"""GPU parity of rows a1-a3: ranking (bit-exact) and the matrix-free H x
against the oracle's explicit sparse H of Eq. (1)."""
import numpy as np
import pytest

from oracle import basis, hamiltonian
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24])
def test_unrank_rank_bit_exact(L):
    hs = need_gpu()
    st_ref = basis.enumerate_states(L)
    with hs.Chain(L, np.zeros(L), sigma=0.0) as c:
        assert c.n == len(st_ref)
        s = c.unrank()
        assert np.array_equal(s.cpu().numpy().astype(np.int64) & ((1 << 32) - 1), st_ref)
        r = c.rank(s)
        assert np.array_equal(r.cpu().numpy(), np.arange(c.n))
        bad = torch.tensor([0, (1 << L) - 1, 1], dtype=torch.int32, device="cuda")
        assert (c.rank(bad).cpu().numpy() == -1).all()


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16, 18])
@pytest.mark.parametrize("shifted", [0, 1])
def test_matvec_f64(L, shifted):
    hs = need_gpu()
    h = inputs.disorder(L, 3.0, 100 + L)
    H, diag, st = hamiltonian.build(L, h)
    sigma = 0.37
    x = inputs.gaussian(len(st), 7)
    ref = H @ x - (sigma * x if shifted else 0)
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(to_dev(x), shifted=bool(shifted)).cpu().numpy()
    scale = np.abs(diag * x).max() + np.abs(x).max() * L
    assert np.abs(y - ref).max() <= 1e-14 * scale


@pytest.mark.parametrize("L", [4, 8, 12, 16, 18])
def test_matvec_f32(L):
    hs = need_gpu()
    h = inputs.disorder(L, 3.0, 200 + L)
    H, diag, st = hamiltonian.build(L, h)
    sigma = -0.2
    x = inputs.gaussian(len(st), 8).astype(np.float32).astype(np.float64)
    ref = H @ x - sigma * x
    absH = abs(H)
    bound = (L + 4) * 2.0 ** -24 * (np.abs(diag - sigma) * np.abs(x) + absH @ np.abs(x)) * 2
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(to_dev(x, torch.float32), shifted=True).cpu().double().numpy()
    assert (np.abs(y - ref) <= bound + 1e-30).all()


def test_diag_and_precond():
    hs = need_gpu()
    L = 12
    h = inputs.disorder(L, 3.0, 5)
    H, diag, st = hamiltonian.build(L, h)
    sigma = 0.11
    with hs.Chain(L, h, sigma=sigma) as c:
        for kind in ("id", "jacobi", "row"):
            d, minv = c.diag(kind)
            m = hamiltonian.precond_diag(H, diag, sigma, kind)
            assert np.abs(d.cpu().numpy() - diag).max() < 1e-13
            # relative error of |a_ii - sigma| grows with the cancellation
            cancel = (np.abs(diag) + abs(sigma) + 1.0) / m
            assert (np.abs(minv.cpu().numpy() * m - 1) <= 4e-16 * cancel * 8).all()


@pytest.mark.parametrize("L", [20, 28])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_matvec_sampled_rows_large(L, dtype):
    """Full-size launch (the configuration the benchmark times), checked on
    sampled rows computed one by one by the oracle from Eq. (1)."""
    hs = need_gpu()
    h = inputs.disorder(L, 3.7, 0)
    n = inputs.dim(L)
    rng = np.random.default_rng(3)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = torch.randn(n, generator=torch.Generator().manual_seed(5), dtype=torch.float64)
    if dtype == "f32":
        x = x.float().double()
    sigma = 0.05
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(x.to(tdt).cuda(), shifted=True).cpu().double().numpy()
    xs = x.numpy()
    rows = np.concatenate([rng.integers(0, n, 300), [0, n - 1, n // 2]])
    for i in rows:
        s = basis.unrank_count(int(i), L)
        d, off = hamiltonian.row(L, h, s, sigma)
        ref = d * xs[i] + sum(v * xs[j] for j, v in off)
        mag = abs(d * xs[i]) + sum(abs(v * xs[j]) for j, v in off)
        tol = (1e-14 if dtype == "f64" else (L + 4) * 2.0 ** -23) * mag + 1e-300
        assert abs(y[i] - ref) <= tol, (i, y[i], ref)
