"""Shared helpers for the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_09732_gb300 import hs
    hs.load()
    return hs


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def fp32_bound(L, x, diag_shifted, rows_abs_sum):
    """Rounding bound of an FP32 row sum with ~L + 2 terms."""
    u = 2.0 ** -24
    return (L + 4) * u * (np.abs(diag_shifted * x) + rows_abs_sum) * 2
