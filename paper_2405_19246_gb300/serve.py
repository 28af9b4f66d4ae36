"""Continuous-batching request loop for MMOT solves on one GPU.

Requests (independent problem instances of any l, N, eps) arrive over time.
The scheduler admits waiting requests, oldest first, as long as their
estimated device memory fits the budget next to the cohorts already running;
every admission forms a cohort: one :class:`~paper_2405_19246_gb300.api.Batch`
on its own CUDA stream, stepped by its own host thread, so cohorts admitted
at different times overlap on the device.  Potentials stay resident in the
cohort's device memory between iterations; after every ``check_every``
iterations the per-instance residuals come back and an instance whose
residual is at most ``tol`` (or whose iteration budget is spent) finishes:
its result is recorded and it stops receiving updates.

Finished instances give their memory back at the next check: when requests
are waiting, the cohort takes the oldest of them that fit into the memory of
its finished instances (plus any unused budget) and re-forms its batch from
its unfinished instances, warm-started from their current potentials
(``Batch.set_potentials``: an instance's Sinkhorn state is its l potentials,
so it continues at an iteration boundary with its iteration count carried
over), and the newly joined requests.  A cohort whose instances have all
finished with no request waiting releases its memory.

The scheduling is host logic; every computation runs in the CUDA library.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    xs: list
    mus: list
    eps: float
    arrival: float = 0.0          # time the request entered the queue
    admitted: float = 0.0
    finished: float = 0.0
    iters: int = 0
    residual: float = float("nan")
    converged: bool = False
    potentials: Optional[list] = None

    @property
    def l(self):
        return len(self.xs)

    @property
    def points(self):
        return sum(len(x) for x in self.xs)

    @property
    def latency(self):
        return self.finished - self.arrival


def estimate_bytes(req: Request, precision: str = "fp32") -> int:
    """Device memory of one instance inside a batch: per point the merged
    stream (position, ln phi, marginal id), potentials, weights and ln
    weights, plus per-tile carries of 2^(l-1) scaled-float states."""
    esz = 4 if precision == "fp32" else 8
    per_point = 2 * esz + 1 + 3 * 8
    tiles = max(1, req.points // 32)
    per_tile = (3 + (req.l - 1)) * (1 << (req.l - 1)) * 2 * esz + 64
    return req.points * per_point + tiles * per_tile


class Cohort:
    """Requests admitted together: one batch, one stream, one stepping thread.

    refill(cohort, freed_bytes) (optional) returns waiting requests that
    join the cohort at a check where some of its instances have finished."""

    def __init__(self, reqs: List[Request], make_batch: Callable, tol: float, itr_max: int,
                 check_every: int, keep_potentials: bool, on_done: Callable,
                 refill: Optional[Callable] = None, precision: str = "fp32"):
        self.reqs = reqs
        self.make_batch = make_batch
        self.tol = tol
        self.itr_max = itr_max
        self.check_every = check_every
        self.keep_potentials = keep_potentials
        self.on_done = on_done
        self.refill = refill
        self.precision = precision
        self.batch = make_batch(reqs)
        self.done = [False] * len(reqs)
        self.base = [0] * len(reqs)   # iterations each request ran before this batch
        self.iters = 0                # iterations of the current batch
        self.released = 0             # finished requests whose memory is not yet reused
        self.regroups = 0
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.error: Optional[BaseException] = None

    def start(self):
        self.thread.start()

    def _finish(self, i, now):
        r = self.reqs[i]
        st = self.batch.status(i)
        r.iters = self.base[i] + (st["iters"] if st["converged"] else self.iters)
        r.residual = st["residual"]
        r.converged = st["converged"]
        if self.keep_potentials:
            r.potentials = [self.batch.get_potentials(i, k) for k in range(r.l)]
        r.finished = now
        self.done[i] = True
        self.released += estimate_bytes(r, self.precision)
        self.on_done(r)

    def _regroup(self, joining: List[Request]):
        """New batch: the unfinished instances, warm-started, then the joining requests."""
        keep = [i for i in range(len(self.reqs)) if not self.done[i]]
        carried = [(self.reqs[i], self.base[i] + self.iters,
                    [self.batch.get_potentials(i, k) for k in range(self.reqs[i].l)]) for i in keep]
        self.batch.close()
        self.batch = None
        reqs = [c[0] for c in carried] + list(joining)
        self.batch = self.make_batch(reqs)
        for i, (_, _, gs) in enumerate(carried):
            for k, g in enumerate(gs):
                self.batch.set_potentials(i, k, g)
        self.reqs = reqs
        self.done = [False] * len(reqs)
        self.base = [c[1] for c in carried] + [0] * len(joining)
        self.iters = 0
        self.released = 0
        self.regroups += 1

    def _loop(self):
        try:
            while not all(self.done):
                self.batch.step(self.check_every, self.tol)
                self.iters += self.check_every
                now = time.perf_counter()
                for i in range(len(self.reqs)):
                    if self.done[i]:
                        continue
                    if self.batch.status(i)["converged"]:
                        self._finish(i, now)
                    elif self.base[i] + self.iters >= self.itr_max:
                        self.batch.freeze(i)
                        self._finish(i, now)
                if self.refill is not None and self.released > 0:
                    joining = self.refill(self, self.released, sum(not d for d in self.done))
                    if joining:
                        self._regroup(joining)
        except BaseException as e:   # surfaced by Server.run
            self.error = e
        finally:
            if self.batch is not None:
                self.batch.close()


class Server:
    """Admit, run and retire requests (see the module docstring).

    make_batch(reqs) builds the device batch of a cohort; the default uses
    :class:`Batch` with a fresh CUDA stream.  mem_budget bounds the estimated
    bytes of all running cohorts; max_cohort bounds the requests per cohort.
    """

    def __init__(self, precision="fp32", tol=1e-6, itr_max=10000, check_every=20,
                 mem_budget=64 << 30, max_cohort=4096, keep_potentials=False, make_batch=None,
                 tick=0.002, tile_caps=None, regroup=True):
        self.precision = precision
        self.tol = tol
        self.itr_max = itr_max
        self.check_every = check_every
        self.mem_budget = mem_budget
        self.max_cohort = max_cohort
        self.keep_potentials = keep_potentials
        self.tick = tick
        self.make_batch = make_batch or self._default_batch
        # optional autotune.TileCapCache: cohorts of a known (l, N, eps)
        # bucket reuse its tuned cap on the points per tile
        self.tile_caps = tile_caps
        self.waiting = collections.deque()
        self.cohorts: List[Cohort] = []
        self.finished: List[Request] = []
        self.used = 0
        self.lock = threading.Lock()
        self.admissions = 0
        # requests that joined a running cohort (its finished instances' memory)
        self.regroup = regroup
        self.joined = 0

    def _default_batch(self, reqs):
        import torch
        from .api import Batch
        stream = torch.cuda.Stream()
        inst = [(r.xs, r.mus, r.eps) for r in reqs]
        tp = self.tile_caps.cap(inst) if self.tile_caps is not None else 0
        return Batch(inst, precision=self.precision, stream=stream, tile_points=tp)

    def submit(self, req: Request, now: Optional[float] = None):
        req.arrival = time.perf_counter() if now is None else now
        with self.lock:
            self.waiting.append(req)

    def _on_done(self, req):
        with self.lock:
            self.finished.append(req)

    def _admit(self):
        """Form one cohort from the oldest waiting requests that fit."""
        take, mem = [], 0
        with self.lock:
            while self.waiting and len(take) < self.max_cohort:
                r = self.waiting[0]
                b = estimate_bytes(r, self.precision)
                if self.used + mem + b > self.mem_budget and (take or self.cohorts):
                    break
                self.waiting.popleft()
                take.append(r)
                mem += b
        if not take:
            return
        now = time.perf_counter()
        for r in take:
            r.admitted = now
        c = Cohort(take, self.make_batch, self.tol, self.itr_max, self.check_every,
                   self.keep_potentials, self._on_done,
                   refill=self._refill if self.regroup else None, precision=self.precision)
        c.mem = mem
        self.used += mem
        self.cohorts.append(c)
        self.admissions += 1
        c.start()

    def _refill(self, cohort, freed, active):
        """Waiting requests, oldest first, that fit into the memory of the
        cohort's finished instances plus the unused budget (called from the
        cohort's thread at a check)."""
        take, mem = [], 0
        with self.lock:
            room = self.mem_budget - self.used + freed
            while self.waiting and active + len(take) < self.max_cohort:
                b = estimate_bytes(self.waiting[0], self.precision)
                if mem + b > room:
                    break
                take.append(self.waiting.popleft())
                mem += b
            if take:
                self.used += mem - freed
                cohort.mem += mem - freed
                self.joined += len(take)
        now = time.perf_counter()
        for r in take:
            r.admitted = now
        return take

    def _reap(self):
        for c in list(self.cohorts):
            if not c.thread.is_alive():
                c.thread.join()
                if c.error is not None:
                    raise c.error
                self.used -= c.mem
                self.cohorts.remove(c)

    def run(self, arrivals=(), until_done=True, timeout=None):
        """Feed (time offset, Request) arrivals in real time and serve until
        every request has finished (or timeout seconds).  Returns the
        finished requests."""
        arrivals = sorted(arrivals, key=lambda a: a[0])
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k][0] <= now:
                self.submit(arrivals[k][1], now=t0 + arrivals[k][0])
                k += 1
            self._reap()
            if self.waiting:
                self._admit()
            if k == len(arrivals) and not self.waiting and not self.cohorts and until_done:
                break
            if timeout is not None and now > timeout:
                break
            time.sleep(self.tick)
        return list(self.finished)


def latency_stats(reqs: List[Request]):
    lat = np.array([r.latency for r in reqs]) if reqs else np.zeros(0)
    return {
        "count": int(lat.size),
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_s": float(lat.mean()) if lat.size else None,
        "converged": int(sum(r.converged for r in reqs)),
    }
