"""GPU parity of the batched disorder sweep (hs_sweep): realisations of two
chain lengths run Algorithm 1 in lockstep rounds, every round's inner solves
(Algorithm 2) in one persistent launch fed by per-length job queues. Each
realisation's K eigenpairs nearest sigma = (E_min + E_max) / 2 against dense
eigh of the oracle's H, its twist overlaps against the oracle's direct sum
(Sec. III), and the realisation averages of |z|^2 (Sec. IV B-C) against the
same averages of the oracle's overlaps."""
import numpy as np
import pytest

from oracle import hamiltonian, twist
from paper_2203_09732_gb300 import inputs
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _realisations(Ls, seed0=100):
    out = []
    for r, L in enumerate(Ls):
        _, h = inputs.disorder_mixed(L, seed0 + r)
        out.append(h)
    return out


def _dense_reference(L, h, K):
    """The K eigenpairs nearest the midpoint of the spectrum (|E - sigma|,
    ties by E), and |z|^2 of each, from dense eigh of the oracle's H."""
    H, diag, states = hamiltonian.build(L, h)
    w, V = np.linalg.eigh(H.toarray())
    sigma = 0.5 * (w[0] + w[-1])
    idx = np.lexsort((w, np.abs(w - sigma)))[:K]
    z = twist.overlap(V[:, idx], states, L)
    return w[idx], np.abs(z) ** 2


@pytest.fixture
def tune_file(tmp_path, monkeypatch):
    p = tmp_path / "tune.json"
    monkeypatch.setenv("HS_SWEEP_TUNE", str(p))
    return p


@pytest.mark.parametrize("form", [None, "2", "1"])
def test_mixed_lengths_against_dense(form, tune_file, monkeypatch):
    """Five realisations at L = 8 and four at L = 10 in one sweep: eigenvalues
    within 1e-10, |z|^2 within 1e-8 per pair, the per-realisation and
    per-length averages of |z|^2 from the same oracle overlaps."""
    hs = need_gpu()
    if form:
        monkeypatch.setenv("HS_SWEEP_FORM", form)
    Ls = [8, 10, 8, 10, 8, 10, 8, 8, 10]
    hl = _realisations(Ls)
    K = 4
    ev, res, z, zz, info = hs.sweep(Ls, hl, K, tol=1e-11)
    assert info["realisations"] == len(Ls) and info["converged"] == len(Ls)
    assert info["nclass"] == 2 and sorted(info["L"]) == [8, 10]
    if form:
        want = hs.FORM_SMEM1 if form == "1" else hs.FORM_SMEM
        assert all(f == want for f in info["form"])
    zz_ref = []
    for r, (L, h) in enumerate(zip(Ls, hl)):
        w_ref, z2_ref = _dense_reference(L, h, K)
        assert np.abs(ev[r] - w_ref).max() < 1e-10, (r, ev[r], w_ref)
        assert np.abs(np.abs(z[r]) ** 2 - z2_ref).max() < 1e-8
        assert res[r].max() < 1e-8
        zz_ref.append(z2_ref.mean())
        assert abs(zz[r] - z2_ref.mean()) < 1e-8
    zz_ref = np.array(zz_ref)
    for c, L in enumerate(info["L"]):
        sel = np.array([x == L for x in Ls])
        assert abs(info["zz_mean"][c] - zz_ref[sel].mean()) < 1e-8
        assert abs(info["zz_std"][c] - zz_ref[sel].std(ddof=1)) < 1e-8


def test_graph_and_eager_rounds_agree(tune_file, monkeypatch):
    """The rounds replayed from the captured graph and launched one by one
    give the same eigenvalues (the same kernels on the same jobs)."""
    hs = need_gpu()
    Ls = [10] * 6
    hl = _realisations(Ls, 200)
    ev1, _, z1, _, i1 = hs.sweep(Ls, hl, 3)
    monkeypatch.setenv("HS_SWEEP_NOGRAPH", "1")
    ev2, _, z2, _, i2 = hs.sweep(Ls, hl, 3)
    assert i2["graph"] == 0
    assert np.abs(ev1 - ev2).max() < 1e-11
    assert np.abs(np.abs(z1) - np.abs(z2)).max() < 1e-9


def test_single_length_matches_lanczos_per_chain(tune_file):
    """One length: the sweep's realisation r equals Chain.eigs with seed + r
    (same start vector, same recurrence): eigenvalues within 1e-11, Lanczos
    rounds = the longest chain's steps."""
    hs = need_gpu()
    L, K, seed = 12, 5, 7
    Ls = [L] * 5
    hl = _realisations(Ls, 300)
    ev, res, z, zz, info = hs.sweep(Ls, hl, K, seed=seed)
    steps = []
    for r, h in enumerate(hl):
        with hs.Chain(L, h) as c:
            e2, v2, r2, i2 = c.eigs(K, seed=seed + r)
        assert np.abs(ev[r] - e2).max() < 1e-11
        steps.append(i2["steps"])
    assert info["rounds"] == max(steps)


def test_schedule_is_cached(tune_file):
    """First call times the schedule and writes the JSON cache; the second
    reads it back (same group size and form)."""
    hs = need_gpu()
    import json
    Ls = [10, 10]
    hl = _realisations(Ls, 400)
    *_, i1 = hs.sweep(Ls, hl, 2)
    assert i1["tuned"] == [1]
    data = json.loads(tune_file.read_text())
    assert len(data) == 1
    entry = next(iter(data.values()))
    assert entry["S"] == i1["S"][0] and entry["S"] >= 1
    *_, i2 = hs.sweep(Ls, hl, 2)
    assert i2["tuned"] == [0] and i2["S"] == i1["S"] and i2["form"] == i1["form"]


def test_forced_group_size(tune_file, monkeypatch):
    """A forced group size (more CTAs per group than needed, so fewer groups
    than realisations: the queue hands several solves to each group)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_SWEEP_S", "40")
    monkeypatch.setenv("HS_SWEEP_FORM", "2")
    Ls = [8] * 7
    hl = _realisations(Ls, 500)
    ev, res, z, zz, info = hs.sweep(Ls, hl, 3, tol=1e-11)
    assert info["S"] == [40] and info["tuned"] == [-1] and info["groups"][0] <= 3
    for r, h in enumerate(hl):
        w_ref, _ = _dense_reference(8, h, 3)
        assert np.abs(ev[r] - w_ref).max() < 1e-10
