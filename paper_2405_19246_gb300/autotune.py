"""Tile-size autotuner for batches of instances.

For a set of instances the tuner builds a batch from a sample of them for
each candidate cap on the points per tile, times a few Sinkhorn iterations
of each (host clock around a synchronised step, which includes the
per-instance residual check), and returns the fastest cap.  Smaller tiles give
more tiles (more parallel work, more carries); larger tiles give fewer,
longer in-tile scans; the best cap depends on the mix of sizes, l and eps.
"""
from __future__ import annotations

import time


def tune_tile_points(instances, precision="fp32", candidates=(0, 1024, 512, 256), sample=64,
                     iters=10, stream=None):
    """Return (best tile_points, {candidate: seconds per iteration})."""
    import torch
    from .api import Batch
    sub = list(instances)[:sample]
    timings = {}
    for tp in candidates:
        with Batch(sub, precision=precision, tile_points=tp, stream=stream) as B:
            B.step(2, 0.0)                       # warm-up (graph capture, operators)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.step(iters, 0.0)
            torch.cuda.synchronize()
            timings[tp] = (time.perf_counter() - t0) / iters
    best = min(timings, key=timings.get)
    return best, timings


def bucket_key(instances):
    """The tuning key of a set of instances: (the most common l, the median
    N as a power-of-two bucket, the median eps in half-decade buckets).
    instances: (xs, mus, eps) triples."""
    import math
    from collections import Counter
    ls = [len(xs) for xs, _, _ in instances]
    Ns = sorted(len(xs[0]) for xs, _, _ in instances)
    es = sorted(float(e) for _, _, e in instances)
    l = Counter(ls).most_common(1)[0][0]
    n_med = Ns[len(Ns) // 2]
    e_med = es[len(es) // 2]
    return (l, int(round(math.log2(max(1, n_med)))), int(math.floor(2.0 * math.log10(e_med))))


class TileCapCache:
    """Tuned tile caps by :func:`bucket_key`: the first set of instances with a
    key is timed (:func:`tune_tile_points`), later sets with the same key
    reuse the cap.  Thread-safe (a serving loop builds cohorts from several
    threads).  tuner(instances) -> (cap, timings) may be replaced (tests)."""

    def __init__(self, tuner=None, **tune_kw):
        import threading
        self.tuner = tuner or (lambda inst: tune_tile_points(inst, **tune_kw))
        self.table = {}
        self.timings = {}
        self.lock = threading.Lock()

    def cap(self, instances):
        key = bucket_key(instances)
        with self.lock:
            if key in self.table:
                return self.table[key]
        best, timings = self.tuner(list(instances))
        with self.lock:
            self.table.setdefault(key, best)
            self.timings.setdefault(key, timings)
            return self.table[key]
