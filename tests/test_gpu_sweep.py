"""GPU parity of the batched disorder sweep (hs_sweep): realisations of two
chain lengths in one persistent launch whose CTA groups take realisations from
per-length queues and run all of Algorithm 1 on each (inner solves by
Algorithm 2) on the device. Each
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


@pytest.mark.parametrize("S", [None, "7"])
def test_mixed_lengths_against_dense(S, tune_file, monkeypatch):
    """Five realisations at L = 8 and four at L = 10 in one sweep (the timed
    group size, and 7 CTAs per group): eigenvalues within 1e-10, |z|^2 within
    1e-8 per pair, the per-realisation and per-length averages of |z|^2 from
    the same oracle overlaps."""
    hs = need_gpu()
    if S:
        monkeypatch.setenv("HS_SWEEP_S", S)
    Ls = [8, 10, 8, 10, 8, 10, 8, 8, 10]
    hl = _realisations(Ls)
    K = 4
    ev, res, z, zz, info = hs.sweep(Ls, hl, K, tol=1e-11)
    assert info["realisations"] == len(Ls) and info["converged"] == len(Ls)
    assert info["nclass"] == 2 and sorted(info["L"]) == [8, 10] and info["launches"] == 1
    if S:
        assert info["S"] == [7, 7] and info["tuned"] == [-1, -1]
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


def test_group_sizes_agree(tune_file, monkeypatch):
    """Groups of 5 and of 19 CTAs (different row partitions, so different
    reduction orders) give the same eigenvalues and overlaps."""
    hs = need_gpu()
    Ls = [12] * 6
    hl = _realisations(Ls, 200)
    monkeypatch.setenv("HS_SWEEP_S", "5")
    ev1, _, z1, _, i1 = hs.sweep(Ls, hl, 3)
    monkeypatch.setenv("HS_SWEEP_S", "19")
    ev2, _, z2, _, i2 = hs.sweep(Ls, hl, 3)
    assert i1["S"] == [5] and i2["S"] == [19]
    assert np.abs(ev1 - ev2).max() < 1e-11
    assert np.abs(np.abs(z1) - np.abs(z2)).max() < 1e-9


def test_single_length_matches_lanczos_per_chain(tune_file):
    """One length: the sweep's realisation r equals Chain.eigs with seed + r
    (same start vector, same recurrence, the convergence test on the device):
    eigenvalues within 1e-11, the longest realisation's Lanczos steps within
    one of the host driver's."""
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
    assert abs(info["max_steps"] - max(steps)) <= 1


def test_schedule_is_cached(tune_file):
    """First call times the schedule and writes the JSON cache; the second
    reads it back (same group size). With fewer realisations than groups, the
    launch uses one group per realisation, at least as large as the timed one."""
    hs = need_gpu()
    import json
    Ls = [10, 10]
    hl = _realisations(Ls, 400)
    *_, i1 = hs.sweep(Ls, hl, 2)
    assert i1["tuned"] == [1]
    data = json.loads(tune_file.read_text())
    assert len(data) == 1
    entry = next(iter(data.values()))
    assert 1 <= entry["S"] <= i1["S"][0] and i1["groups"][0] >= len(Ls)
    *_, i2 = hs.sweep(Ls, hl, 2)
    assert i2["tuned"] == [0] and i2["S"] == i1["S"]


def test_forced_group_size(tune_file, monkeypatch):
    """A forced group size (more CTAs per group than needed, so fewer groups
    than realisations: the queue hands several solves to each group)."""
    hs = need_gpu()
    monkeypatch.setenv("HS_SWEEP_S", "40")
    Ls = [8] * 7
    hl = _realisations(Ls, 500)
    ev, res, z, zz, info = hs.sweep(Ls, hl, 3, tol=1e-11)
    assert info["S"] == [40] and info["tuned"] == [-1] and info["groups"][0] <= 3
    for r, h in enumerate(hl):
        w_ref, _ = _dense_reference(8, h, 3)
        assert np.abs(ev[r] - w_ref).max() < 1e-10
