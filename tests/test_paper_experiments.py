"""The paper's 1-D experiments (Sec. 5.1 random weights, Sec. 5.2 Ricker
wavelets) on the CPU side: why the re-centred (log-domain) form is needed.

Sec. 5.2 (Fig. 2b) reports that without log-domain stabilisation the method
stops early on the Ricker problem at N = 100, eps = 1e-3 (the iterates leave
the floating-point range).  The literal, unstabilised Algorithm 4 of the
oracle (FS-3 with FTVP-1, plain scalings phi = 1/N at the start) breaks down
the same way on our reading of that problem (uniform grid on [-2, 2],
tau = 0, 0.75, 1.5, delta = 1e-3, L = N): its scalings overflow and the
stopping residual becomes NaN within a few hundred iterations, while at
eps = 0.1 it runs to the end.  The GPU side of the same experiments is in
``tests/test_gpu_paper_experiments.py``.
"""
import numpy as np

import oracle
from paper_2405_19246_gb300 import workloads as wl


def _fs3(N, eps, iters):
    xs, mus = wl.paper_ricker(N)
    h = float(xs[0][1] - xs[0][0])
    return oracle.fs3(mus[0], mus[1], mus[2], h, eps, 0.0, iters)


def _finite(r):
    return all(np.all(np.isfinite(r[k])) for k in ("phi", "psi", "varphi"))


def test_unstabilised_algorithm4_overflows_on_ricker_at_small_eps():
    r = _fs3(100, 1e-3, 300)
    assert not _finite(r)
    assert r["iters"] < 300          # the NaN residual ends the loop early
    assert not np.isfinite(r["res"])


def test_unstabilised_algorithm4_runs_at_the_default_eps():
    r = _fs3(100, 1e-1, 300)
    assert _finite(r)
    assert r["iters"] == 300
    assert 0.0 < r["res"] < 1e-2
