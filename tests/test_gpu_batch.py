"""GPU parity of batches of independent instances.

A batch lays instances with the same l out one after another; no state may
cross an instance boundary and every instance keeps its own eps.  Each
instance of a batch must therefore give what the same instance gives alone
(a single-instance plan, same iteration count), within the FP32 / FP64
tolerances, and what the oracle gives.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import api as A
    return A


def _mixed_instances(count, seed, N_range=(40, 900), eps_range=(5e-3, 1e-1), l_range=(2, 8)):
    params = wl.batched_instance_params(count, seed_cfg=seed, l_range=l_range, N_range=N_range,
                                        eps_range=eps_range)
    inst = []
    for i, (l, N, eps) in enumerate(params):
        xs, mus = wl.batched_instance(i, l, int(N), seed_cfg=seed)
        inst.append((xs, mus, eps))
    return inst


TOL_G = {"fp32": 2e-4, "fp64": 1e-9}   # potentials after a few iterations, in units of eps


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_iterations_match_single_instances(api, prec):
    inst = _mixed_instances(24, seed=901)
    n_it = 4
    with api.Batch(inst, precision=prec) as B:
        assert B.info()["groups"] >= 5
        B.step(n_it, 0.0)
        for i, (xs, mus, eps) in enumerate(inst):
            with api.Plan(xs, mus, eps, precision=prec) as P:
                P.sinkhorn_step(n_it)
                for k in range(len(xs)):
                    d = np.max(np.abs(B.get_potentials(i, k) - P.get_potentials(k))) / eps
                    assert d <= TOL_G[prec], (i, k, d)


def test_batch_matches_oracle(api):
    inst = _mixed_instances(10, seed=902, N_range=(30, 300), l_range=(2, 5))
    n_it = 3
    with api.Batch(inst, precision="fp64") as B:
        B.step(n_it, 0.0)
        for i, (xs, mus, eps) in enumerate(inst):
            gs = [np.full(len(x), -eps * math.log(len(x))) for x in xs]
            for _ in range(n_it):
                for j in range(len(xs)):
                    gs[j] = oracle.potential_update(mus[j], oracle.marginal_subset(xs, gs, eps, j), eps)
            for k in range(len(xs)):
                d = np.max(np.abs(B.get_potentials(i, k) - gs[k])) / eps
                assert d <= 1e-9, (i, k, d)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_solve_stops_each_instance(api, prec):
    """Each instance stops at the first check with residual <= tol; its result
    equals the same instance run alone for the same number of iterations."""
    inst = _mixed_instances(16, seed=903, N_range=(40, 400), eps_range=(3e-2, 1e-1), l_range=(2, 6))
    tol = 1e-6 if prec == "fp64" else 1e-5
    with api.Batch(inst, precision=prec) as B:
        res = B.solve(tol, 3000, check_every=5)
        iters = [r["iters"] for r in res]
        assert len(set(iters)) > 1          # instances stop at different checks
        for i, (xs, mus, eps) in enumerate(inst):
            st = B.status(i)
            assert st["converged"] and st["residual"] <= tol, (i, st)
            assert iters[i] % 5 == 0
            with api.Plan(xs, mus, eps, precision=prec) as P:
                out = P.solve(0.0, iters[i])
                for k in range(len(xs)):
                    d = np.max(np.abs(B.get_potentials(i, k) - P.get_potentials(k))) / eps
                    assert d <= 50 * TOL_G[prec], (i, k, d)
                if len(xs) < 8:
                    assert abs(res[i]["W"] - out["W"]) <= 1e-4 * abs(out["W"]), (i, res[i]["W"], out["W"])
                assert abs(res[i]["mass"] - out["mass"]) <= 1e-5


def test_frozen_instance_keeps_its_potentials(api):
    inst = _mixed_instances(8, seed=904, N_range=(40, 300), eps_range=(2e-2, 1e-1), l_range=(3, 6))
    with api.Batch(inst, precision="fp32") as B:
        B.step(3, 0.0)
        r = np.array([B.status(i)["residual"] for i in range(len(inst))])
        tol = float(np.median(r))
        B.step(0, tol)       # no iteration: freezes the instances at or below the median
        frozen = [B.status(i)["converged"] for i in range(len(inst))]
        assert 0 < sum(frozen) < len(inst)
        before = [[B.get_potentials(i, k) for k in range(len(inst[i][0]))] for i in range(len(inst))]
        B.step(4, 0.0)
        for i in range(len(inst)):
            for k in range(len(inst[i][0])):
                g = B.get_potentials(i, k)
                if frozen[i]:
                    np.testing.assert_array_equal(g, before[i][k])
                else:
                    assert np.max(np.abs(g - before[i][k])) > 0.0


def test_instance_result_is_independent_of_its_neighbours(api):
    """The same instance in two different batches gives the same potentials."""
    inst = _mixed_instances(12, seed=905, N_range=(40, 600), l_range=(3, 6))
    other = _mixed_instances(12, seed=906, N_range=(40, 600), l_range=(3, 6))
    mix = other[:5] + [inst[3]] + other[5:]
    with api.Batch(inst, precision="fp32") as A, api.Batch(mix, precision="fp32") as B:
        A.step(6, 0.0)
        B.step(6, 0.0)
        xs, mus, eps = inst[3]
        for k in range(len(xs)):
            d = np.max(np.abs(A.get_potentials(3, k) - B.get_potentials(5, k))) / eps
            assert d <= TOL_G["fp32"], (k, d)


def test_served_result_same_alone_and_in_mix(api):
    """A request served alone and the same request served among others
    (other cohorts overlapping on the device) give the same result."""
    from paper_2405_19246_gb300.serve import Request, Server
    inst = _mixed_instances(10, seed=907, N_range=(40, 400), eps_range=(3e-2, 1e-1), l_range=(3, 7))

    def req(i):
        xs, mus, eps = inst[i]
        return Request(rid=i, xs=xs, mus=mus, eps=eps)

    alone = Server(tol=1e-5, itr_max=4000, check_every=10, keep_potentials=True).run([(0.0, req(4))])
    mix = Server(tol=1e-5, itr_max=4000, check_every=10, keep_potentials=True, max_cohort=3, regroup=False)
    res = {r.rid: r for r in mix.run([(0.005 * i, req(i)) for i in range(10)])}
    a, m = alone[0], res[4]
    assert len(res) == 10 and mix.admissions >= 2
    assert a.converged and m.converged and a.iters == m.iters
    eps = inst[4][2]
    for k in range(len(inst[4][0])):
        d = np.max(np.abs(a.potentials[k] - m.potentials[k])) / eps
        assert d <= 2e-4, (k, d)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_warm_start_continues_the_run(api, prec):
    """Potentials of an instance moved into another batch (set_potentials on
    all l marginals) continue its run: a few more iterations there give what
    the original batch gives."""
    # one l, so the moved instance shares its launch group with instances of
    # other eps and is not the group's first
    inst = _mixed_instances(4, seed=908, N_range=(40, 500), eps_range=(2e-2, 1e-1), l_range=(4, 4))
    other = _mixed_instances(5, seed=909, N_range=(40, 500), eps_range=(2e-2, 1e-1), l_range=(4, 4))
    q, j = 2, 3
    with api.Batch(inst, precision=prec) as A:
        A.step(5, 0.0)
        gs = [A.get_potentials(q, k) for k in range(len(inst[q][0]))]
        with api.Batch(other[:j] + [inst[q]] + other[j:], precision=prec) as B:
            assert B.info()["groups"] == 1
            for k, g in enumerate(gs):
                B.set_potentials(j, k, g)
            for k, g in enumerate(gs):
                np.testing.assert_array_equal(B.get_potentials(j, k), g)
            A.step(4, 0.0)
            B.step(4, 0.0)
            eps = inst[q][2]
            for k in range(len(gs)):
                d = np.max(np.abs(A.get_potentials(q, k) - B.get_potentials(j, k))) / eps
                assert d <= TOL_G[prec], (k, d)


def test_set_potentials_reactivates_and_rejects_nan(api):
    inst = _mixed_instances(6, seed=910, N_range=(40, 300), eps_range=(2e-2, 1e-1), l_range=(3, 5))
    with api.Batch(inst, precision="fp32") as B:
        B.step(2, 0.0)
        B.freeze(1)
        g = B.get_potentials(1, 0)
        bad = g.copy()
        bad[len(bad) // 2] = np.nan
        with pytest.raises(Exception):
            B.set_potentials(1, 0, bad)
        np.testing.assert_array_equal(B.get_potentials(1, 0), g)
        B.set_potentials(1, 0, g)
        before = B.get_potentials(1, 1)
        B.step(2, 0.0)
        assert np.max(np.abs(B.get_potentials(1, 1) - before)) > 0.0   # updated again


def test_served_requests_join_a_running_cohort(api):
    """A memory budget of two and a half requests of one size: two start,
    the rest join the running cohort as its instances finish; every request
    converges and matches the same request solved alone."""
    from paper_2405_19246_gb300.serve import Request, Server, estimate_bytes
    inst = _mixed_instances(6, seed=911, N_range=(200, 200), eps_range=(3e-2, 1e-1), l_range=(4, 4))

    def req(i):
        xs, mus, eps = inst[i]
        return Request(rid=i, xs=xs, mus=mus, eps=eps)

    budget = int(2.5 * max(estimate_bytes(req(i)) for i in range(6)))
    srv = Server(tol=1e-5, itr_max=4000, check_every=10, keep_potentials=True, mem_budget=budget)
    res = {r.rid: r for r in srv.run([(0.0, req(i)) for i in range(6)])}
    assert len(res) == 6 and all(r.converged for r in res.values())
    assert srv.joined >= 1
    for i in (0, 5):
        a = Server(tol=1e-5, itr_max=4000, check_every=10, keep_potentials=True).run([(0.0, req(i))])[0]
        m = res[i]
        assert abs(a.iters - m.iters) <= 10, (i, a.iters, m.iters)
        eps = inst[i][2]
        for k in range(len(inst[i][0])):
            d = np.max(np.abs(a.potentials[k] - m.potentials[k])) / eps
            assert d <= 1e-3, (i, k, d)
