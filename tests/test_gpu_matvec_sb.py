"""GPU parity of the superblock forms of H x (row a3 for long chains): the
matrix-free (H - sigma) x of Eq. (1) with the x tiles of two superblocks
staged in shared memory, against the oracle's explicit sparse H and against
the block form. Two superblock forms: four low bits with one lane per
sub-block (sb4; the FP64 default, HS_SB4=1 forces it) and ten low bits with
one warp per sub-block (the FP32 default, HS_SB4=0 forces it)."""
import numpy as np
import pytest

from oracle import basis, hamiltonian
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["1", "0"])
@pytest.mark.parametrize("L", [22, 24])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shifted", [0, 1])
def test_superblock_matvec_vs_oracle(L, dtype, shifted, form, monkeypatch):
    """Every row against the explicit matrix (sb4: 14-bit windows in FP32,
    13-bit in FP64; ten-bit form: 12-bit windows at L = 22, 14/13-bit at 24)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_HV_SB", "1")
    monkeypatch.setenv("HS_SB4", form)
    h = inputs.disorder(L, 3.0, 300 + L)
    H, diag, st = hamiltonian.build(L, h)
    sigma = 0.41
    x = inputs.gaussian(len(st), 17 + L)
    tdt = torch.float64
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
        tdt = torch.float32
    ref = H @ x - (sigma * x if shifted else 0)
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(to_dev(x, tdt), shifted=bool(shifted)).cpu().double().numpy()
    if dtype == "f64":
        scale = np.abs(diag * x).max() + np.abs(x).max() * L
        assert np.abs(y - ref).max() <= 1e-14 * scale
    else:
        s = sigma if shifted else 0.0
        bound = (L + 4) * 2.0 ** -24 * (np.abs(diag - s) * np.abs(x) + abs(H) @ np.abs(x)) * 2
        assert (np.abs(y - ref) <= bound + 1e-30).all()


@pytest.mark.parametrize("form", ["1", "0"])
@pytest.mark.parametrize("L", [24, 26, 28])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_superblock_matches_block_form(L, dtype, form, monkeypatch):
    """Full-size launches: superblock form against the block (gather) form on
    the same x; the two differ only in the order of the row sums."""
    hs = need_gpu()
    monkeypatch.setenv("HS_SB4", form)
    h = inputs.disorder(L, 3.7, 4)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    with hs.Chain(L, h, sigma=0.1) as c:
        x = torch.randn(c.n, generator=torch.Generator().manual_seed(2), dtype=torch.float64).to(tdt).cuda()
        monkeypatch.setenv("HS_HV_SB", "0")
        y0 = c.matvec(x, shifted=True)
        monkeypatch.setenv("HS_HV_SB", "1")
        y1 = c.matvec(x, shifted=True)
        torch.cuda.synchronize()
    assert bool(torch.isfinite(y1).all())
    scale = float(x.abs().max()) * (L + 3.7 * L)
    tol = (1e-14 if dtype == "f64" else (L + 4) * 2.0 ** -23) * scale
    assert float((y1 - y0).abs().max()) <= tol


@pytest.mark.parametrize("form", ["1", "0"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("offset", [1, 3])
def test_superblock_unaligned_vectors(dtype, offset, form, monkeypatch):
    """x and y that start off a 16-byte boundary (views at an element offset):
    the staged copies and the stores follow the vectors, and the result is
    the same as with aligned vectors, element for element, with nothing
    written outside y."""
    hs = need_gpu()
    monkeypatch.setenv("HS_HV_SB", "1")
    monkeypatch.setenv("HS_SB4", form)
    L = 24
    h = inputs.disorder(L, 3.0, 8)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    with hs.Chain(L, h, sigma=0.3) as c:
        x = torch.randn(c.n, generator=torch.Generator().manual_seed(6), dtype=torch.float64).to(tdt).cuda()
        y = c.matvec(x, shifted=True)
        xb = torch.zeros(c.n + 8, dtype=tdt, device="cuda")
        yb = torch.full((c.n + 8,), float("nan"), dtype=tdt, device="cuda")
        xb[offset:offset + c.n] = x
        c.matvec(xb[offset:offset + c.n], y=yb[offset:offset + c.n], shifted=True)
        torch.cuda.synchronize()
    assert torch.equal(yb[offset:offset + c.n], y)
    assert bool(torch.isnan(yb[:offset]).all()) and bool(torch.isnan(yb[offset + c.n:]).all())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_four_bit_form_sampled_rows_l28(dtype, monkeypatch):
    """L = 28 (40,116,600 rows), the size of the benchmark, through the
    four-low-bit form in FP32 and FP64: 300 sampled rows computed one by one
    from Eq. (1)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_HV_SB", "1")
    monkeypatch.setenv("HS_SB4", "1")
    L = 28
    h = inputs.disorder(L, 3.7, 0)
    n = inputs.dim(L)
    rng = np.random.default_rng(28)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = torch.randn(n, generator=torch.Generator().manual_seed(3), dtype=torch.float64).to(tdt)
    sigma = 0.07
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(x.cuda(), shifted=True).cpu().double().numpy()
    xs = x.double().numpy()
    for i in np.concatenate([rng.integers(0, n, 300), [0, n - 1]]):
        s = basis.unrank_count(int(i), L)
        d, off = hamiltonian.row(L, h, s, sigma)
        ref = d * xs[i] + sum(v * xs[j] for j, v in off)
        mag = abs(d * xs[i]) + sum(abs(v * xs[j]) for j, v in off)
        tol = 1e-14 * mag if dtype == "f64" else (L + 4) * 2.0 ** -23 * mag
        assert abs(y[i] - ref) <= tol + 1e-300, (i, y[i], ref)


def test_superblock_sampled_rows_l26(monkeypatch):
    """L = 26 (10,400,600 rows; FP64 plan: 4096 pairs of 13-bit superblocks):
    sampled rows computed one by one from Eq. (1)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_HV_SB", "1")
    L = 26
    h = inputs.disorder(L, 3.7, 1)
    n = inputs.dim(L)
    rng = np.random.default_rng(4)
    x = torch.randn(n, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    sigma = -0.15
    with hs.Chain(L, h, sigma=sigma) as c:
        y = c.matvec(x.cuda(), shifted=True).cpu().numpy()
    xs = x.numpy()
    for i in np.concatenate([rng.integers(0, n, 200), [0, n - 1]]):
        s = basis.unrank_count(int(i), L)
        d, off = hamiltonian.row(L, h, s, sigma)
        ref = d * xs[i] + sum(v * xs[j] for j, v in off)
        mag = abs(d * xs[i]) + sum(abs(v * xs[j]) for j, v in off)
        assert abs(y[i] - ref) <= 1e-14 * mag + 1e-300, (i, y[i], ref)


@pytest.mark.parametrize("dtype,es", [("f32", 4), ("f64", 8)])
def test_matvec_rejects_vectors_off_element_alignment(dtype, es):
    """A device pointer that is not a multiple of the element size is refused
    on the host with HS_BAD_ARG, before any launch; the handle stays usable."""
    import ctypes
    hs = need_gpu()
    L = 24
    tdt = torch.float64 if dtype == "f64" else torch.float32
    with hs.Chain(L, inputs.disorder(L, 1.0, 2), sigma=0.0) as c:
        x = torch.randn(c.n + 2, dtype=tdt, device="cuda")
        y = torch.zeros(c.n + 2, dtype=tdt, device="cuda")
        dt = hs.F64 if dtype == "f64" else hs.F32
        for dx, dy in ((es // 2, 0), (0, es // 2)):
            st = c._lib.hs_matvec(c._hd, ctypes.c_void_p(x.data_ptr() + dx),
                                  ctypes.c_void_p(y.data_ptr() + dy), dt, 1)
            assert st == hs.HS_BAD_ARG
        assert float(y.abs().max()) == 0.0
        y1 = c.matvec(x[:c.n], shifted=True)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(y1).all())
