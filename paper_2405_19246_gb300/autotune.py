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
