"""Host-side logic of the benchmark's multi-GPU mode (replicas, no data-path
collective), exercised as two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [i for s in range(3) for i in bench.rank_realisations(rank, world, s, 8)]
    got = [None] * world
    dist.all_gather_object(got, mine)
    # each rank times its own steps; the job time is the maximum over ranks
    t = torch.tensor([1.5 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, got, float(t.item())))
    dist.destroy_process_group()


def test_two_ranks_get_disjoint_realisations_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, tmax in res:
        a, b = set(got[0]), set(got[1])
        assert not (a & b)
        assert len(a) == len(got[0]) == 24
        assert tmax == 2.5


def test_realisations_follow_the_sweep_recipe():
    sys.path.insert(0, ROOT)
    import bench
    h, seed, hv = bench.realisation(3, 16)
    assert 0.5 <= h <= 6.0 and len(hv) == 16 and (abs(hv) <= h).all()
    assert bench.realisation(3, 16)[2].tolist() == hv.tolist()


class _FakeChain:
    def __init__(self):
        self.share = None
        self.history = []

    def set_sm_budget(self, n):
        self.share = n
        self.history.append(n)


@pytest.mark.parametrize("static", [False, True])
def test_sm_shares_never_oversubscribe_and_pass_on(static):
    """The benchmark's SM shares: 24 realisations on 152 SMs start on 6 each.
    As they finish (in a random order, from many threads), the ones still
    running get the freed SMs, up to the cap; at no time do the shares of the
    running realisations sum to more than the SM count. With static shares
    nothing changes."""
    import random
    import threading
    import time
    sys.path.insert(0, ROOT)
    import bench

    nsm, B = 152, 24
    base = nsm // B
    chains = {i: _FakeChain() for i in range(B)}
    worst = []

    class Checked(bench.Shares):
        def _check(self):
            tot = sum(chains[k].share for k in self.live)
            worst.append(tot)
            assert tot <= self.nsm
            for k in self.live:
                assert self.base <= chains[k].share <= max(self.base, self.cap)

        def start(self, key, chain):
            super().start(key, chain)
            with self.lock:
                self._check()

        def done(self, key):
            super().done(key)
            with self.lock:
                self._check()

    shares = Checked(B, base, nsm, static=static)
    for i in range(B):
        shares.start(i, chains[i])
    order = list(range(B))
    random.Random(7).shuffle(order)
    errors = []

    def finish(i, delay):
        try:
            time.sleep(delay)
            shares.done(i)
        except AssertionError as e:  # pragma: no cover - reported below
            errors.append(e)

    th = [threading.Thread(target=finish, args=(i, 0.002 * r)) for r, i in enumerate(order)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    assert max(worst) <= nsm
    last = chains[order[-1]]
    if static:
        assert all(c.history == [base] for c in chains.values())
    else:
        # the last realisation ends up with the cap; shares only ever grow
        assert last.share == min(bench.SHARE_CAP, nsm)
        for c in chains.values():
            assert c.history == sorted(c.history)
