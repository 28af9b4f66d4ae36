"""The paper's 1-D experiments on the GPU path.

* Tables 1 and 2 (Sec. 5.1 random weights on a uniform grid of [0, 1],
  Sec. 5.2 Ricker wavelets on [-2, 2]): l = 3, eps = 0.1, 100 Sinkhorn
  iterations; the plan of the fast method P_O against the plan of the dense
  Sinkhorn P_S (products over the full N^3 tensor, ``oracle.brute``), in the
  Frobenius norm, for N = 10 .. 160 (Ricker up to 80).  The paper reports about 1e-16.  Here
  the all-FP64 GPU path must stay below 1e-14 and the FP32-scan path below
  1e-5 ||P_S||_F (its products carry a relative error up to 1e-5, which
  moves each potential by at most that much times eps per update).
* Fig. 2b (Sec. 5.2, N = 100, eps = 1e-3): the re-centred form runs 300
  iterations with finite potentials and the same residual as the oracle's
  log-domain Sinkhorn, where the unstabilised Algorithm 4 overflows
  (``tests/test_paper_experiments.py``).
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Plan():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300.api import Plan as P
    return P


def _dense_plan(xs, gs, eps):
    return brute.plan(xs, gs, eps)


def _problem(kind, N):
    return wl.paper_random_1d(N) if kind == "random" else wl.paper_ricker(N)


@pytest.fixture(scope="module")
def dense_runs():
    out = {}
    for kind in ("random", "ricker"):
        for N in (10, 20, 40, 80, 160):
            if kind == "ricker" and N == 160:
                continue   # the dense N^3 Sinkhorn takes about a minute at N = 160
            xs, mus = _problem(kind, N)
            gs = brute.sinkhorn_dense(xs, mus, 0.1, 100)
            out[(kind, N)] = (xs, mus, _dense_plan(xs, gs, 0.1))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,N", [("random", 10), ("random", 20), ("random", 40), ("random", 80),
                                    ("random", 160), ("ricker", 10), ("ricker", 20), ("ricker", 40),
                                    ("ricker", 80)])
def test_fast_plan_equals_dense_sinkhorn_plan(Plan, dense_runs, prec, kind, N):
    xs, mus, PS = dense_runs[(kind, N)]
    p = Plan(xs, mus, 0.1, precision=prec)
    p.sinkhorn_step(100)
    gs = [p.get_potentials(k) for k in range(3)]
    p.close()
    PO = _dense_plan(xs, gs, 0.1)
    d = float(np.linalg.norm((PO - PS).ravel()))
    bound = 1e-14 if prec == "fp64" else 1e-5 * float(np.linalg.norm(PS.ravel()))
    assert d <= bound, (prec, kind, N, d)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ricker_small_eps_runs_where_the_unstabilised_form_overflows(Plan, prec):
    N, eps, iters = 100, 1e-3, 300
    xs, mus = wl.paper_ricker(N)
    p = Plan(xs, mus, eps, precision=prec)
    res = p.sinkhorn_step(iters, residual=True)
    gs = [p.get_potentials(k) for k in range(3)]
    p.close()
    assert all(np.all(np.isfinite(g)) for g in gs)
    ref = oracle.sinkhorn(xs, mus, eps, 0.0, iters)
    assert np.isfinite(ref["res"])
    assert abs(res - ref["res"]) <= (1e-9 if prec == "fp64" else 1e-4) * max(ref["res"], 1e-6), (res, ref["res"])
