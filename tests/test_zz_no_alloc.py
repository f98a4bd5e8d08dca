"""hs_twist_noalloc, the entry point for callers that cannot allocate device
memory (code inside another component's stream capture, plug-ins whose host
application owns every device allocation). It must give the same twist
overlaps as hs_twist, call after call, while using only its fixed static
scratch. Kept in a file that pytest collects last."""
import numpy as np
import pytest

from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,ka,kb", [(12, 3, 5), (16, 3, 5), (24, 8, 2)])
def test_matches_hs_twist_on_two_calls(L, ka, kb):
    """L = 24 (n = 2.7M) fills the 256-CTA grid, so the last-CTA reduction
    adds 256 partial rows and threads unrank starting ranks in the millions;
    K = 8 is the most vectors the scratch holds."""
    hs = need_gpu()
    n = inputs.dim(L)
    psi_a = to_dev(inputs.gaussian(n, 31, count=ka))
    psi_b = to_dev(inputs.gaussian(n, 32, count=kb))
    with hs.Chain(L, np.zeros(L), sigma=0.0) as c:
        ref_a = c.twist(psi_a)
        ref_b = c.twist(psi_b)
    stream = torch.cuda.current_stream()
    for psi, ref in ((psi_a, ref_a), (psi_b, ref_b)):
        z = torch.full((2 * psi.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        assert hs.twist_noalloc(L, psi, z, stream) == hs.HS_OK
        stream.synchronize()
        zz = z.cpu().numpy()
        got = zz[0::2] + 1j * zz[1::2]
        scale = (psi.double() ** 2).sum(dim=1).max().item()
        assert np.abs(got - ref).max() <= 1e-12 * scale


def test_rejects_more_vectors_than_the_scratch_holds():
    hs = need_gpu()
    L = 8
    psi = torch.zeros((9, inputs.dim(L)), dtype=torch.float64, device="cuda")
    z = torch.zeros(18, dtype=torch.float64, device="cuda")
    assert hs.twist_noalloc(L, psi, z) == hs.HS_BAD_ARG
    assert hs.twist_noalloc(7, psi[:2], z) == hs.HS_BAD_ARG
