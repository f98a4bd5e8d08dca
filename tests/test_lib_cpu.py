"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/hs.h declares; host-only entry points work without a GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_09732_gb300 import build, hs
    build.build()
    return hs.load()


def test_exports_every_declared_symbol(lib):
    from paper_2203_09732_gb300 import hs
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(hs.SYMBOLS) == decl


def test_tridiag_eig_matches_numpy(lib):
    from paper_2203_09732_gb300 import hs
    rng = np.random.default_rng(0)
    for k in (1, 2, 3, 10, 57, 130):
        a = rng.standard_normal(k)
        b = rng.standard_normal(k - 1)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        th, Y = hs.tridiag_eig(a, b)
        w, V = np.linalg.eigh(T)
        assert np.abs(th - w).max() < 1e-12 * max(1, np.abs(w).max())
        assert np.abs(T @ Y - Y * th).max() < 1e-11
        assert np.abs(Y.T @ Y - np.eye(k)).max() < 1e-12


def test_tridiag_eig_degenerate(lib):
    from paper_2203_09732_gb300 import hs
    a = np.array([1.0, 1.0, 1.0, 2.0])
    b = np.array([0.0, 0.0, 1e-300])
    th = hs.tridiag_eig(a, b, vectors=False)
    assert np.allclose(th, [1, 1, 1, 2])


def test_create_rejects_bad_arguments_without_gpu(lib):
    import ctypes
    from paper_2203_09732_gb300 import hs
    h = np.zeros(33)
    hd = ctypes.c_void_p()
    for L in (2, 3, 5, 34, 0):
        st = lib.hs_create(L, h.ctypes.data_as(hs.c_dp), 0.0, None, ctypes.byref(hd))
        assert st == hs.HS_BAD_ARG
    hn = np.array([0.0, np.nan, 0.0, 0.0])
    st = lib.hs_create(4, hn.ctypes.data_as(hs.c_dp), 0.0, None, ctypes.byref(hd))
    assert st == hs.HS_BAD_ARG
    assert lib.hs_last_error(None) == b"null handle"


def test_binding_fails_loudly_without_library(tmp_path):
    """No CPU fallback: a missing libhs.so is an error, not a silent path."""
    import importlib
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import os; os.environ['HS_LIB_PATH'] = %r\n"
            "from paper_2203_09732_gb300 import hs\n"
            "try:\n    hs.load()\nexcept RuntimeError as e:\n    print('raised', e)\n") % (
        ROOT, str(tmp_path / "missing.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "raised" in r.stdout and "missing" in r.stdout


def test_level_ratio_matches_oracle(lib):
    """hs_level_ratio (host-only) against the oracle's r_k, on random levels,
    an unsorted input and the equal-spacing case."""
    from oracle import observables as ob
    from paper_2203_09732_gb300 import hs
    rng = np.random.default_rng(5)
    for K in (3, 4, 17, 50):
        e = rng.normal(size=K)
        r, mean = hs.level_ratio(e)
        ref = ob.level_spacing_ratios(e)
        assert np.allclose(r, ref, rtol=0, atol=1e-15) and abs(mean - ref.mean()) < 1e-15
    r, mean = hs.level_ratio(np.arange(6.0))
    assert np.all(r == 1.0) and mean == 1.0
    with pytest.raises(hs.HSError):
        hs.level_ratio([0.0, 1.0])


def test_sym_eigvals_matches_numpy(lib):
    """The host step of hs_entanglement: Householder + implicit QL eigenvalues
    of symmetric matrices against numpy's eigvalsh (random, rank-deficient like
    a reduced density matrix, diagonal, 1 x 1)."""
    from paper_2203_09732_gb300 import hs
    rng = np.random.default_rng(7)
    for n in (1, 2, 3, 10, 70, 200):
        A = rng.normal(size=(n, n))
        A = A + A.T
        w = hs.sym_eigvals(A)
        assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 1e-12 * max(1.0, np.abs(A).sum(axis=1).max())
        B = rng.normal(size=(n, max(1, n // 3)))
        R = B @ B.T
        w = hs.sym_eigvals(R)
        assert np.abs(w - np.linalg.eigvalsh(R)).max() <= 1e-12 * max(1.0, np.trace(R))
    D = np.diag([3.0, -1.0, 2.0])
    assert np.allclose(hs.sym_eigvals(D), [-1.0, 2.0, 3.0], atol=1e-15)


def test_sweep_rejects_bad_arguments(lib):
    """hs_sweep checks its arguments before any device work: no realisation,
    three chain lengths, an odd L."""
    import ctypes
    from paper_2203_09732_gb300 import hs
    info = hs.SweepInfo()
    ev = np.zeros(8)
    for Ls in ([], [8, 10, 12], [9]):
        B = len(Ls)
        Larr = (ctypes.c_int * max(B, 1))(*(Ls or [8]))
        h = np.zeros(max(sum(Ls), 1))
        st = lib.hs_sweep(B, Larr, h.ctypes.data_as(hs.c_dp), 2, 0, 1e-10, 0, 1e-12, 2,
                          ev.ctypes.data_as(hs.c_dp), None, None, None, ctypes.byref(info))
        assert st == hs.HS_BAD_ARG
