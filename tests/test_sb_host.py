"""CPU check of the superblock H x arithmetic (row a3 for long chains).

The kernel's plan builder and its per-lane and per-phase row code live in the
package's sb.cuh as host/device functions. tests/host/sb_host_check.cu runs
them on the CPU in the kernel's order, with NaN in every staged buffer and
around x, and the result is compared here with the oracle's explicit sparse H
of Eq. (1): every row, FP64 and FP32, over splits (L, k, KS) that reach every
bond kind, including the windows the library picks at L = 22 and 24 and
degenerate ones (one or two mid bits, two top bits)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hamiltonian
from paper_2203_09732_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("sbhost") / "sb_host_check"
    src = os.path.join(HERE, "host", "sb_host_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-o", str(out), src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(out)


# (L, k, KS): KS - k mid bits, L - KS top bits
SPLITS = [(12, 4, 8), (12, 2, 4), (14, 4, 6), (16, 5, 10), (18, 6, 12), (20, 8, 12),
          (20, 10, 16), (22, 10, 11), (22, 10, 12), (24, 10, 13), (24, 10, 14)]


@pytest.mark.parametrize("L,k,KS", SPLITS)
def test_superblock_rows_vs_explicit_matrix(checker, tmp_path, L, k, KS):
    h = np.asarray(inputs.disorder(L, 3.0, 7 * L + k), dtype=np.float64)
    H, diag, st = hamiltonian.build(L, h)
    x = inputs.gaussian(len(st), 11 + L)
    h.tofile(tmp_path / "h.bin")
    x.tofile(tmp_path / "x.bin")
    sigma = 0.37
    ref = H @ x - sigma * x
    x32 = x.astype(np.float32).astype(np.float64)
    ref32 = H @ x32 - sigma * x32
    bound32 = (L + 4) * 2.0 ** -24 * (np.abs(diag - sigma) * np.abs(x32) + abs(H) @ np.abs(x32)) * 2
    scale = np.abs(diag * x).max() + np.abs(x).max() * L
    for shift in (0, 3):
        r = subprocess.run([checker, str(L), str(k), str(KS), repr(sigma), str(shift), str(tmp_path)],
                           capture_output=True, text=True)
        assert r.returncode == 0, (r.stdout, r.stderr)
        y64 = np.fromfile(tmp_path / "y64.bin")
        y32 = np.fromfile(tmp_path / "y32.bin")
        assert np.isfinite(y64).all() and np.isfinite(y32).all()
        assert np.abs(y64 - ref).max() <= 1e-14 * scale
        assert (np.abs(y32 - ref32) <= bound32 + 1e-30).all()
    # preconditioner entries of the MINRES row passes (Sec. II, Eq. (rownorm)
    # and M_Jacobi) against the oracle's, row by row
    mrow = np.fromfile(tmp_path / "mrow.bin")
    mjac = np.fromfile(tmp_path / "mjac.bin")
    mrow32 = np.fromfile(tmp_path / "mrow32.bin")
    ref_row = hamiltonian.precond_diag(H, diag, sigma, "row")
    ref_jac = np.abs(diag - sigma)
    assert np.abs(mrow - ref_row).max() <= 1e-14 * ref_row.max()
    assert np.abs(mjac - ref_jac).max() <= 1e-14 * (np.abs(diag).max() + 1)
    # FP32: a_ii - sigma from FP32 terms of magnitude up to |a_ii| + L, then
    # one square root
    assert (np.abs(mrow32 - ref_row) <= 2.0 ** -22 * (np.abs(diag) + L + 1)).all()


def test_plan_rejects_splits_out_of_range(checker, tmp_path):
    """More than 8 mid bits, or fewer than two top bits: no plan (the library
    then uses the block form)."""
    L = 16
    inputs_h = np.asarray(inputs.disorder(L, 1.0, 1), dtype=np.float64)
    inputs_h.tofile(tmp_path / "h.bin")
    for (k, KS) in ((2, 14), (4, 15), (10, 16)):
        r = subprocess.run([checker, str(L), str(k), str(KS), "0.0", "0", str(tmp_path)],
                           capture_output=True, text=True)
        assert r.returncode == 4 and "does not apply" in r.stdout


@pytest.fixture(scope="module")
def checker4(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = tmp_path_factory.mktemp("sb4host") / "sb4_host_check"
    src = os.path.join(HERE, "host", "sb4_host_check.cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-o", str(out), src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(out)


# (L, KS) with k = 4 low bits: KS - 4 mid bits, L - KS top bits; the library's
# window at L >= 22 is KS = 14 (FP32) and 13 (FP64)
SPLITS4 = [(12, 5), (12, 8), (14, 6), (14, 10), (16, 8), (16, 12), (18, 13), (18, 14), (20, 14),
           (22, 13), (22, 14), (24, 14)]


@pytest.mark.parametrize("L,KS", SPLITS4)
def test_four_bit_superblock_rows_vs_explicit_matrix(checker4, tmp_path, L, KS):
    """The lane-per-sub-block row code: every row against the oracle's explicit
    H in FP64 (1e-14) and FP32 (the rounding bound of an FP32 row sum), with NaN
    in every slot element, G entry and guard element that the kernel must not
    read."""
    h = np.asarray(inputs.disorder(L, 3.0, 5 * L + KS), dtype=np.float64)
    H, diag, st = hamiltonian.build(L, h)
    x = inputs.gaussian(len(st), 3 + L)
    h.tofile(tmp_path / "h.bin")
    x.tofile(tmp_path / "x.bin")
    sigma = -0.29
    ref = H @ x - sigma * x
    x32 = x.astype(np.float32).astype(np.float64)
    ref32 = H @ x32 - sigma * x32
    bound32 = (L + 4) * 2.0 ** -24 * (np.abs(diag - sigma) * np.abs(x32) + abs(H) @ np.abs(x32)) * 2
    scale = np.abs(diag * x).max() + np.abs(x).max() * L
    r = subprocess.run([checker4, str(L), str(KS), repr(sigma), str(tmp_path)],
                       capture_output=True, text=True)
    assert r.returncode == 0, (r.stdout, r.stderr)
    y64 = np.fromfile(tmp_path / "y64.bin")
    y32 = np.fromfile(tmp_path / "y32.bin")
    assert np.isfinite(y64).all() and np.isfinite(y32).all()
    assert np.abs(y64 - ref).max() <= 1e-14 * scale
    assert (np.abs(y32 - ref32) <= bound32 + 1e-30).all()


def test_four_bit_plan_rejects_splits_out_of_range(checker4, tmp_path):
    """More than 10 mid bits, or fewer than two top bits: no plan."""
    L = 18
    np.asarray(inputs.disorder(L, 1.0, 1), dtype=np.float64).tofile(tmp_path / "h.bin")
    for KS in (4, 15, 17):
        r = subprocess.run([checker4, str(L), str(KS), "0.0", str(tmp_path)],
                           capture_output=True, text=True)
        assert r.returncode == 4 and "does not apply" in r.stdout
