"""GPU parity: the CUDA marginal products and Sinkhorn iterations against the
CPU oracle on the same seeded inputs, element by element.

Tolerances (relative error of M_j, i.e. absolute error of ln M_j): 1e-5 for
the FP32 scans, 1e-12 for the all-FP64 path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def Plan():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300.api import Plan as P
    return P


def _init_g(xs, eps):
    return [np.full(len(x), -eps * math.log(len(x))) for x in xs]


def _rand_g(xs, eps, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    return [(-eps * math.log(len(x)) + scale * rng.normal(size=len(x))) for x in xs]


def _lnM_err(got, ref):
    both_inf = np.isneginf(got) & np.isneginf(ref)
    d = np.where(both_inf, 0.0, np.abs(got - ref))
    return float(np.max(d)) if d.size else 0.0


CASES = [
    # l, N per marginal, eps, ties, zeros
    (2, 5000, 1e-2, False, False),
    (3, 3000, 1e-2, False, False),
    (3, 2500, 5e-3, True, False),
    (4, 2100, 1e-3, False, False),
    (4, 1700, 2e-2, True, True),
    (5, 900, 1e-2, False, True),
    (6, 300, 3e-2, False, False),
    (7, 150, 5e-2, False, False),
    (8, 90, 5e-2, False, False),
]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps,ties,zeros", CASES)
def test_marginal_product_parity(Plan, prec, l, N, eps, ties, zeros):
    Ns = [N + 37 * k for k in range(l)]   # ragged sizes, several tiles and a tail
    xs, mus = wl.random_small(l, Ns, seed=100 + l, ties=ties, zeros=zeros, grid=N // 3)
    gs = _rand_g(xs, eps, seed=l)
    plan = Plan(xs, mus, eps, precision=prec)
    for k in range(l):
        plan.set_potentials(k, gs[k])
    assert plan.info()["tiles"] >= 2
    for j in range(l):
        ref = oracle.marginal_subset(xs, gs, eps, j)
        got = plan.marginal(j, "lnM")
        assert _lnM_err(got, ref) <= TOL[prec], (j, _lnM_err(got, ref))
    plan.close()


# sparse supports at small eps: neighbouring points lie tens of eps apart, so
# states of one subset level differ by far more than the FP32 range
SPARSE = [(4, 69, 1.2e-3, 176), (5, 160, 1.33e-3, 107), (6, 154, 1.27e-3, 255),
          (7, 78, 1.46e-3, 49), (8, 82, 2.8e-3, 119), (3, 64, 1e-3, 7)]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps,inst", SPARSE)
def test_sparse_supports_small_eps(Plan, prec, l, N, eps, inst):
    xs, mus = wl.batched_instance(inst, l, N)
    gs = _init_g(xs, eps)
    plan = Plan(xs, mus, eps, precision=prec)
    for it in range(3):
        for j in range(l):
            ref = oracle.marginal_subset(xs, gs, eps, j)
            got = plan.marginal(j, "lnM")
            # a log value of magnitude L carries a rounding error of order u L;
            # decay exponents reach w_max x/eps (w_max = floor(l/2) ceil(l/2))
            tol = TOL[prec] * max(1.0, 1e-2 * float(np.max(np.abs(ref))))
            if prec == "fp64":
                tol += 8 * 1.1e-16 * (l // 2) * ((l + 1) // 2) * max(float(np.max(x)) for x in xs) / eps
            assert _lnM_err(got, ref) <= tol, (it, j, _lnM_err(got, ref))
            gs[j] = oracle.potential_update(mus[j], ref, eps)
            plan.set_potentials(j, gs[j])
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tiny_sparse_random(Plan, prec):
    """Many tiny instances whose points lie tens to hundreds of eps apart:
    every carry crosses a wide gap and each tile holds one to three points."""
    rng = np.random.default_rng(2024)
    worst = 0.0
    for trial in range(150):
        l = int(rng.integers(2, 7))
        N = int(rng.integers(2, 9))
        eps = float(10 ** rng.uniform(-3, -1.5))
        xs = [np.sort(rng.random(N)) for _ in range(l)]
        mus = [np.full(N, 1.0 / N) for _ in range(l)]
        gs = _rand_g(xs, eps, seed=trial, scale=2 * eps)
        plan = Plan(xs, mus, eps, precision=prec)
        for k in range(l):
            plan.set_potentials(k, gs[k])
        for j in range(l):
            ref = oracle.marginal_subset(xs, gs, eps, j)
            err = _lnM_err(plan.marginal(j, "lnM"), ref)
            worst = max(worst, err)
            assert err <= TOL[prec] * max(1.0, 1e-2 * float(np.max(np.abs(ref)))), (trial, l, N, eps, j, err)
        plan.close()


OBJ_TOL = {"fp32": 2e-5, "fp64": 1e-11}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps,ties,zeros", CASES)
def test_objective_parity(Plan, prec, l, N, eps, ties, zeros):
    """W = <C, T> (gap formula over all 2^l subsets), mass, primal and dual
    terms for random potentials against the oracle's all-subset sweep."""
    Ns = [N + 37 * k for k in range(l)]
    xs, mus = wl.random_small(l, Ns, seed=300 + l, ties=ties, zeros=zeros, grid=N // 3)
    gs = _rand_g(xs, eps, seed=50 + l)
    plan = Plan(xs, mus, eps, precision=prec)
    for k in range(l):
        plan.set_potentials(k, gs[k])
    got = plan.objective()
    lnM, lnZ, W = oracle.allpass(xs, gs, eps)
    marg = [np.exp(gs[k] / eps + lnM[k]) for k in range(l)]
    Z = math.exp(lnZ)
    primal = sum(float(np.dot(gs[k], marg[k])) for k in range(l))
    dual = sum(float(np.dot(gs[k], mus[k])) for k in range(l)) + eps - eps * Z
    res = sum(float(np.sum(np.abs(marg[k] - mus[k]))) for k in range(l))
    tol = OBJ_TOL[prec]
    assert abs(got["W"] - W) <= tol * abs(W), (got["W"], W)
    assert abs(got["mass"] - Z) <= tol * Z, (got["mass"], Z)
    scale = sum(float(np.dot(np.abs(gs[k]), marg[k])) for k in range(l))
    assert abs(got["primal"] - primal) <= tol * scale, (got["primal"], primal)
    assert abs(got["dual"] - dual) <= tol * (scale + eps), (got["dual"], dual)
    assert abs(got["residual"] - res) <= tol * (res + Z), (got["residual"], res)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_solve_objective_matches_oracle_sinkhorn(Plan, prec):
    """A short solve (20 iterations, l = 3): W, residual and mass against the
    oracle's log-domain Sinkhorn run from the same start."""
    xs, mus = wl.sorted_uniform_lognormal(l=3, N=1500, instance=9)
    eps = 2e-2
    ref = oracle.sinkhorn(xs, mus, eps, tol=0.0, itr_max=20)
    plan = Plan(xs, mus, eps, precision=prec)
    out = plan.solve(0.0, 20)
    tol = 1e-4 if prec == "fp32" else 1e-9
    assert abs(out["W"] - ref["W"]) <= tol * abs(ref["W"]), (out["W"], ref["W"])
    assert abs(out["mass"] - ref["mass"]) <= tol, (out["mass"], ref["mass"])
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sinkhorn_iterations_parity(Plan, prec):
    xs, mus = wl.sorted_uniform_lognormal(l=4, N=2000, instance=3)
    eps = 5e-3
    n_it = 5
    plan = Plan(xs, mus, eps, precision=prec)
    plan.sinkhorn_step(n_it)
    gs = _init_g(xs, eps)
    for _ in range(n_it):
        for j in range(4):
            gs[j] = oracle.potential_update(mus[j], oracle.marginal_subset(xs, gs, eps, j), eps)
    for j in range(4):
        g = plan.get_potentials(j)
        # potential errors accumulate over iterations; compare in units of eps
        err = float(np.max(np.abs(g - gs[j]))) / eps
        assert err <= 50 * TOL[prec], (j, err)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_grid_mixture_c1_full_run(Plan, prec):
    """l = 3, N = 1000 uniform grid, eps = 1e-2, 200 iterations (literal
    Algorithm 4 in the oracle) against the GPU path."""
    xs, mus = wl.uniform_grid_mixture(l=3, N=1000)
    eps, iters = 1e-2, 200
    r = oracle.fs3(*mus, h=1.0 / 999, eps=eps, tol=0.0, itr_max=iters)
    plan = Plan(xs, mus, eps, precision=prec)
    out = plan.solve(0.0, iters)
    assert out["iters"] == iters
    gref = [eps * np.log(r["phi"]), eps * np.log(r["psi"]), eps * np.log(r["varphi"])]
    for j in range(3):
        err = float(np.max(np.abs(plan.get_potentials(j) - gref[j]))) / eps
        assert err <= (1e-3 if prec == "fp32" else 1e-9), (j, err)
    plan.close()


def test_updated_marginal_is_exact(Plan):
    xs, mus = wl.sorted_uniform_lognormal(l=3, N=4000, instance=5)
    eps = 1e-2
    plan = Plan(xs, mus, eps, precision="fp32")
    plan.sinkhorn_step(2)
    marg = plan.marginal(2, "plan")
    # the last marginal was updated last: it matches mu_3 up to the FP32 tolerance
    np.testing.assert_allclose(marg, mus[2], rtol=1e-5, atol=0)
    plan.close()


def test_edge_sizes(Plan):
    # single-point marginals, l = 2 and l = 3
    for l in (2, 3):
        xs = [np.array([0.1 * (k + 1)]) for k in range(l)]
        mus = [np.array([1.0]) for _ in range(l)]
        for prec in ("fp32", "fp64"):
            plan = Plan(xs, mus, 0.05, precision=prec)
            gs = _init_g(xs, 0.05)
            for j in range(l):
                ref = oracle.marginal_subset(xs, gs, 0.05, j)
                assert _lnM_err(plan.marginal(j, "lnM"), ref) <= TOL[prec]
            plan.close()


def test_all_points_coincide(Plan):
    # every support point at the same coordinate: only ties
    l, N = 4, 700
    xs = [np.full(N + k, 0.5) for k in range(l)]
    mus = [np.full(N + k, 1.0 / (N + k)) for k in range(l)]
    gs = _init_g(xs, 0.1)
    plan = Plan(xs, mus, 0.1, precision="fp32")
    for j in range(l):
        assert _lnM_err(plan.marginal(j, "lnM"), oracle.marginal_subset(xs, gs, 0.1, j)) <= 1e-5
    plan.close()


def test_invalid_inputs(Plan):
    from paper_2405_19246_gb300._native import MmotError
    x = np.linspace(0, 1, 10)
    m = np.full(10, 0.1)
    with pytest.raises(MmotError, match="UNSORTED"):
        Plan([x, x[::-1].copy()], [m, m], 0.1)
    with pytest.raises(MmotError, match="INVALID_ARG"):
        Plan([x, x], [m, m * 2], 0.1)
    with pytest.raises(MmotError, match="INVALID_ARG"):
        Plan([x, x], [m, m], -1.0)
    with pytest.raises(MmotError, match="INVALID_ARG"):
        Plan([x] * 9, [m] * 9, 0.1)
