"""Host logic of the continuous-batching server (no GPU): admission by
memory budget in arrival order, cohort retirement, iteration budgets and
latency bookkeeping, with a stand-in for the device batch."""
import threading
import time

import numpy as np

from paper_2405_19246_gb300.serve import Request, Server, estimate_bytes, latency_stats


class FakeBatch:
    """Instance i converges after need[i] iterations (residual 1/(1+iters)).
    Its "potentials" carry (rid, iterations run so far), so a warm start
    through set_potentials resumes its progress."""

    live = 0
    peak = 0
    created = 0
    lock = threading.Lock()

    def __init__(self, reqs, need):
        self.reqs = reqs
        self.need = [need[r.rid] for r in reqs]
        self.it = 0
        self.offset = [0] * len(reqs)
        self.frozen = [False] * len(reqs)
        self.conv = [False] * len(reqs)
        self.conv_it = [0] * len(reqs)
        with FakeBatch.lock:
            FakeBatch.live += 1
            FakeBatch.created += 1
            FakeBatch.peak = max(FakeBatch.peak, FakeBatch.live)

    def step(self, n, tol):
        time.sleep(0.001)
        self.it += n
        for i, nd in enumerate(self.need):
            if not self.conv[i] and not self.frozen[i] and self.offset[i] + self.it >= nd:
                self.conv[i] = True
                self.conv_it[i] = self.it
        return sum(not (c or f) for c, f in zip(self.conv, self.frozen))

    def status(self, i):
        it = self.conv_it[i] if self.conv[i] else self.it
        return dict(iters=it, residual=1.0 / (1 + it), converged=self.conv[i])

    def freeze(self, i):
        self.frozen[i] = True

    def get_potentials(self, i, k):
        return np.array([float(self.reqs[i].rid), float(self.offset[i] + self.it)])

    def set_potentials(self, i, k, g):
        assert g[0] == self.reqs[i].rid
        self.offset[i] = int(g[1])

    def close(self):
        with FakeBatch.lock:
            FakeBatch.live -= 1


def _reqs(n, N=100, l=3):
    return [Request(rid=i, xs=[np.zeros(N)] * l, mus=[np.zeros(N)] * l, eps=0.1) for i in range(n)]


def test_all_requests_finish_in_budget_and_order():
    reqs = _reqs(40)
    need = {r.rid: 20 * (1 + r.rid % 5) for r in reqs}
    FakeBatch.peak = 0
    per = estimate_bytes(reqs[0])
    srv = Server(check_every=10, itr_max=1000, mem_budget=4 * per, max_cohort=3,
                 make_batch=lambda rs: FakeBatch(rs, need), keep_potentials=True, regroup=False)
    arrivals = [(0.0005 * i, r) for i, r in enumerate(reqs)]
    done = srv.run(arrivals)
    assert len(done) == 40 and all(r.converged for r in done)
    # a cohort holds at most 3 requests and at most 4 requests' memory runs at once
    assert srv.admissions >= 14
    assert FakeBatch.peak <= 4
    # admission follows arrival order
    adm = sorted(reqs, key=lambda r: r.admitted)
    assert [r.rid for r in adm] == sorted(r.rid for r in adm)
    # each result belongs to its request; iterations are the ones that converged it
    for r in done:
        assert r.potentials[0][0] == r.rid
        assert r.iters == need[r.rid]
        assert r.finished >= r.admitted >= r.arrival


def test_finished_instances_make_room_for_waiting_requests():
    """With regrouping, waiting requests join the running cohort as its
    instances finish; unfinished instances continue from their potentials
    with their iteration counts carried over."""
    reqs = _reqs(12)
    need = {r.rid: (40 if r.rid % 3 else 130) for r in reqs}
    FakeBatch.peak = 0
    FakeBatch.created = 0
    per = estimate_bytes(reqs[0])
    srv = Server(check_every=10, itr_max=1000, mem_budget=4 * per, max_cohort=4,
                 make_batch=lambda rs: FakeBatch(rs, need), keep_potentials=True)
    done = srv.run([(0.0, r) for r in reqs])
    assert len(done) == 12 and all(r.converged for r in done)
    # one cohort: everything after the first four joined it as room appeared
    assert srv.admissions == 1 and srv.joined == 8
    assert FakeBatch.peak == 1 and FakeBatch.created > 1
    assert srv.used == 0
    for r in done:
        assert r.iters == need[r.rid]
        assert r.potentials[0][0] == r.rid and r.potentials[0][1] == need[r.rid]
    adm = sorted(reqs, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in adm] == sorted(r.rid for r in adm)


def test_regrouped_requests_keep_their_iteration_budget():
    reqs = _reqs(6)
    need = {r.rid: (20 if r.rid < 3 else 10 ** 9) for r in reqs}
    per = estimate_bytes(reqs[0])
    srv = Server(check_every=10, itr_max=60, mem_budget=4 * per, max_cohort=4,
                 make_batch=lambda rs: FakeBatch(rs, need))
    done = srv.run([(0.0, r) for r in reqs])
    assert len(done) == 6 and srv.joined == 2
    for r in done:
        assert r.converged == (r.rid < 3)
        assert r.iters == (20 if r.rid < 3 else 60)


def test_iteration_budget_ends_unconverged_requests():
    reqs = _reqs(6)
    need = {r.rid: (30 if r.rid % 2 else 10 ** 9) for r in reqs}
    srv = Server(check_every=10, itr_max=50, make_batch=lambda rs: FakeBatch(rs, need))
    done = srv.run([(0.0, r) for r in reqs])
    assert len(done) == 6
    for r in done:
        assert r.converged == bool(r.rid % 2)
        assert r.iters == (30 if r.rid % 2 else 50)
    st = latency_stats(done)
    assert st["count"] == 6 and st["converged"] == 3 and st["p99_s"] >= st["p50_s"] > 0


def test_oversized_request_runs_alone():
    reqs = _reqs(3, N=10 ** 6, l=6)
    need = {r.rid: 10 for r in reqs}
    FakeBatch.peak = 0
    srv = Server(check_every=10, mem_budget=1, make_batch=lambda rs: FakeBatch(rs, need))
    done = srv.run([(0.0, r) for r in reqs])
    assert len(done) == 3 and FakeBatch.peak == 1


def test_tile_cap_cache_tunes_each_bucket_once():
    from paper_2405_19246_gb300.autotune import TileCapCache, bucket_key
    calls = []

    def tuner(inst):
        calls.append(len(inst))
        return 512, {0: 2.0, 512: 1.0}

    def inst(l, N, eps):
        return ([np.zeros(N)] * l, [np.full(N, 1.0 / N)] * l, eps)

    cache = TileCapCache(tuner=tuner)
    a = [inst(4, 1000, 1e-2), inst(4, 1100, 1.2e-2), inst(3, 900, 1e-2)]
    b = [inst(4, 1050, 1.1e-2), inst(4, 1000, 1e-2)]
    c = [inst(4, 1000, 1e-3)]
    assert bucket_key(a) == (4, 10, -4) and bucket_key(b) == bucket_key(a)
    assert bucket_key(c) != bucket_key(a)
    assert cache.cap(a) == 512 and cache.cap(b) == 512 and calls == [3]
    assert cache.cap(c) == 512 and calls == [3, 1]


def test_refill_respects_cohort_size_and_budget():
    """Joins take waiting requests oldest first, at most up to max_cohort
    active instances and within the freed memory plus the unused budget;
    the server's and the cohort's memory accounting follow."""
    import collections
    reqs = _reqs(6)
    per = estimate_bytes(reqs[0])
    srv = Server(check_every=10, mem_budget=5 * per, max_cohort=4,
                 make_batch=lambda rs: FakeBatch(rs, {r.rid: 10 for r in rs}))

    class C:
        mem = 4 * per

    srv.used = 4 * per
    srv.waiting = collections.deque(reqs)
    # one instance finished (its memory freed), three still active: one joins
    take = srv._refill(C, per, 3)
    assert [r.rid for r in take] == [0]
    assert srv.used == 4 * per and C.mem == 4 * per and srv.joined == 1
    # two finished, two active: room for 2 + 1 unused, but the cohort caps at 4
    srv.used = 4 * per
    C.mem = 4 * per
    take = srv._refill(C, 2 * per, 2)
    assert [r.rid for r in take] == [1, 2]
    assert srv.used == 4 * per and C.mem == 4 * per
    # nothing freed, budget full: nobody joins
    srv.used = 5 * per
    assert srv._refill(C, 0, 1) == []
    assert [r.rid for r in srv.waiting] == [3, 4, 5]
