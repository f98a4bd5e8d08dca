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
