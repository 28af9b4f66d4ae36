"""Shards of one instance on one GPU with the host exchange, against the CPU
oracle and against one plan of the whole instance.

* The shard operator (``mmot_shard_operator``) of tiny shards against the
  brute-force sum over placements (``oracle.brute.range_operator``).
* Products of every marginal through P = 2, 3, 4 shards (each holding many
  tiles, so the entering states pass through every chunk of the carry scan)
  against the oracle's subset chains, element by element.
* Three Gauss-Seidel iterations through the shards against the same
  iterations of one plan, and the stopping residual (Algorithm 1).

Tolerances as for every product test: 1e-5 on ln M in FP32, 1e-12 in FP64
(scaled by the magnitude of the log values, a log-domain value of magnitude L
carrying a rounding error of order u L).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def sh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import shard
    return shard


def _tol(prec, ref):
    fin = ref[np.isfinite(ref)]
    return TOL[prec] * max(1.0, 1e-2 * float(np.max(np.abs(fin)))) if fin.size else TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,n", [(2, 6), (3, 6), (4, 5), (5, 4)])
def test_shard_operator_matches_brute_force(sh, prec, l, n):
    rng = np.random.default_rng(100 + l)
    eps = 0.2
    N = 3 * n
    xs = [np.sort(rng.random(N)) for _ in range(l)]
    mus = [np.full(N, 1.0 / N) for _ in range(l)]
    gs = [0.3 * eps * rng.standard_normal(N) - eps * math.log(N) for _ in range(l)]
    parts = sh.split(xs, mus, 3)
    X, K, I = brute.merged_order(xs)
    lo = 0
    for xq, mq in parts:
        hi = lo + sum(len(x) for x in xq)
        p = sh.ShardPlan(xq, mq, [N] * l, eps, prec)
        # this shard's potentials: the points of each marginal inside [lo, hi)
        for k in range(l):
            idx = I[lo:hi][K[lo:hi] == k]
            p.set_potentials(k, gs[k][idx])
        x_L, x_R = p.ends
        assert x_L == X[lo] and x_R == X[hi - 1]
        for j in range(l):
            got = p.operator(j)
            for d in range(2):
                ref = brute.range_operator(xs, gs, eps, j, lo, hi, x_L, x_R, backward=(d == 1))
                fin = np.isfinite(ref)
                assert np.array_equal(np.isfinite(got[d]), fin), (j, d, got[d], ref)
                err = float(np.max(np.abs(got[d][fin] - ref[fin])))
                assert err <= _tol(prec, ref[fin]), (prec, j, d, err)
        p.close()
        lo = hi


@pytest.fixture(scope="module")
def problem4():
    l, N, eps = 4, 20000, 5e-3
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=31)
    rng = np.random.default_rng(31)
    gs = [-eps * math.log(N) + 0.4 * eps * rng.standard_normal(N) for _ in range(l)]
    refs = [oracle.marginal_subset(xs, gs, eps, j) for j in range(l)]
    return dict(xs=xs, mus=mus, gs=gs, eps=eps, refs=refs)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("P", [2, 3, 4])
def test_sharded_products_match_oracle(sh, problem4, prec, P):
    R = problem4
    S = sh.ShardedPlan(R["xs"], R["mus"], R["eps"], P, precision=prec)
    for k in range(4):
        S.set_potentials(k, R["gs"][k])
    for j in range(4):
        got = S.marginal(j, "lnM")
        ref = R["refs"][j]
        err = float(np.max(np.abs(got - ref)))
        assert err <= _tol(prec, ref), (prec, P, j, err)
    S.close()


def test_sharded_products_many_tiles(sh):
    """l = 3, 3 x 300000 points in two shards of several hundred tiles each."""
    l, N, eps = 3, 300000, 2e-3
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=32)
    rng = np.random.default_rng(32)
    gs = [-eps * math.log(N) + 0.3 * eps * rng.standard_normal(N) for _ in range(l)]
    S = sh.ShardedPlan(xs, mus, eps, 2, precision="fp32")
    for k in range(l):
        S.set_potentials(k, gs[k])
    for j in (0, 2):
        ref = oracle.marginal_subset(xs, gs, eps, j)
        got = S.marginal(j, "lnM")
        assert float(np.max(np.abs(got - ref))) <= _tol("fp32", ref), j
    S.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps,P", [(3, 5000, 1e-2, 2), (4, 4000, 5e-3, 3), (5, 2500, 1e-2, 2)])
def test_sharded_iterations_match_single_plan(sh, prec, l, N, eps, P):
    from paper_2405_19246_gb300.api import Plan
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=40 + l)
    one = Plan(xs, mus, eps, precision=prec)
    r1 = one.sinkhorn_step(3, residual=True)
    S = sh.ShardedPlan(xs, mus, eps, P, precision=prec)
    rS = S.sinkhorn_step(3, residual=True)
    for k in range(l):
        a, b = S.get_potentials(k), one.get_potentials(k)
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        err = float(np.max(np.abs(a[fin] - b[fin]))) / eps
        assert err <= 40 * _tol(prec, b[fin] / eps), (prec, k, err)
    assert abs(rS - r1) <= 1e-4 * max(r1, 1e-3) if prec == "fp32" else abs(rS - r1) <= 1e-9 * max(r1, 1e-3)
    # the residual is Algorithm 1's over marginals 1..l-1: recompute with the oracle
    gs = [S.get_potentials(k) for k in range(l)]
    ref = 0.0
    for k in range(l - 1):
        lnM = oracle.marginal_subset(xs, gs, eps, k)
        ref += float(np.sum(np.abs(np.exp(gs[k] / eps + lnM) - mus[k])))
    assert abs(rS - ref) <= (2e-4 if prec == "fp32" else 1e-9) * max(ref, 1e-3), (rS, ref)
    one.close()
    S.close()


def test_shard_calls_reject_misuse(sh):
    from paper_2405_19246_gb300 import _native as nat
    from paper_2405_19246_gb300.api import Plan
    xs, mus = wl.sorted_uniform_lognormal(l=3, N=500, instance=5)
    p = Plan(xs, mus, 1e-2)
    with pytest.raises(nat.MmotError, match="not a shard plan"):
        nat.check(nat.lib().mmot_shard_update(p._h, 0))
    p.close()
    parts = sh.split(xs, mus, 2)
    s = sh.ShardPlan(parts[0][0], parts[0][1], [500] * 3, 1e-2)
    with pytest.raises(nat.MmotError, match="no inflow"):
        s.update(1)
    with pytest.raises(nat.MmotError, match="shard plans iterate"):
        nat.check(nat.lib().mmot_sinkhorn_step(s._h, 1, None))
    bad = np.zeros(4)
    bad[2] = np.nan
    with pytest.raises(nat.MmotError, match="not finite"):
        s.set_inflow(0, bad, None)
    s.close()
    xs6, mus6 = wl.sorted_uniform_lognormal(l=6, N=50, instance=5)
    with pytest.raises(nat.MmotError) as ei:
        sh.ShardPlan(xs6, mus6, [50] * 6, 1e-2)
    assert ei.value.status == 8   # MMOT_ERR_RANGE
