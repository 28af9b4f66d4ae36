"""GPU parity at the sizes the benchmark runs, element by element against the
CPU oracle (the fast product is exact, Sec. 4.2; Table `table1` reports the
fast and dense plans agreeing to about 1e-16).

* The benchmark workload itself: l = 4, N = 2^20 sorted U[0,1] points per
  marginal, LogNormal(0,1) weights, eps = 1e-3.  All four products from
  phi = 1/N, the potentials after two Gauss-Seidel iterations, the stopping
  residual of Algorithm 1 (marginals 1..l-1) and the objective terms.
* More tiles than one block of the carry scan takes (l = 3, N = 12e6).
* l = 8 at N = 2^16: many warp tiles, several chunks per level scan.
* The stopping residual for l = 3, 5, 8.

Tolerances (absolute error of ln M, i.e. relative error of M): 1e-5 for the
FP32 scans, 1e-12 for the all-FP64 path, widened for log values of magnitude
L by max(1, L/100) and, in FP64, by the rounding of decay exponents up to
w_max x/eps (8 u w_max max(x)/eps): a log-domain value of magnitude L carries
a rounding error of order u L.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
U64 = 1.1102230246251565e-16


@pytest.fixture(scope="module")
def Plan():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300.api import Plan as P
    return P


def _init_g(xs, eps):
    return [np.full(len(x), -eps * math.log(len(x))) for x in xs]


def _tol(prec, ref, xs, eps, l):
    t = TOL[prec] * max(1.0, 1e-2 * float(np.max(np.abs(ref[np.isfinite(ref)]))))
    if prec == "fp64":
        t += 8 * U64 * (l // 2) * ((l + 1) // 2) * max(float(np.max(np.abs(x))) for x in xs) / eps
    return t


def _lnM_err(got, ref):
    both_inf = np.isneginf(got) & np.isneginf(ref)
    d = np.where(both_inf, 0.0, np.abs(got - ref))
    return float(np.max(d)) if d.size else 0.0


def _residual(xs, mus, gs, eps, ks):
    """Algorithm 1's stopping test: sum over marginals ks of ||phi_k M_k - mu_k||_1,
    with M_k from the oracle; also returns sum of the plan marginals (scale)."""
    res, scale = 0.0, 0.0
    for k in ks:
        lnM = oracle.marginal_subset(xs, gs, eps, k)
        with np.errstate(invalid="ignore"):
            a = gs[k] / eps + lnM
        marg = np.where(np.isneginf(gs[k]) | np.isneginf(lnM), 0.0, np.exp(a))
        res += float(np.sum(np.abs(marg - mus[k])))
        scale += float(np.sum(marg))
    return res, scale


# ---- the benchmark workload: l = 4, N = 2^20, eps = 1e-3 -------------------

C2 = dict(l=4, N=1 << 20, eps=1e-3)


@pytest.fixture(scope="module")
def c2_ref():
    l, N, eps = C2["l"], C2["N"], C2["eps"]
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=0)
    g0 = _init_g(xs, eps)
    lnM0 = [oracle.marginal_subset(xs, g0, eps, j) for j in range(l)]
    gs = [g.copy() for g in g0]
    for _ in range(2):
        for j in range(l):
            gs[j] = oracle.potential_update(mus[j], oracle.marginal_subset(xs, gs, eps, j), eps)
    return dict(xs=xs, mus=mus, g0=g0, lnM0=lnM0, g2=gs)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c2_products_from_initial_potentials(Plan, c2_ref, prec):
    xs, eps, l = c2_ref["xs"], C2["eps"], C2["l"]
    plan = Plan(xs, c2_ref["mus"], eps, precision=prec)
    info = plan.info()
    assert info["total_points"] == l * C2["N"]
    assert info["tiles"] >= 1024, info
    for j in range(l):
        ref = c2_ref["lnM0"][j]
        got = plan.marginal(j, "lnM")
        err = _lnM_err(got, ref)
        assert err <= _tol(prec, ref, xs, eps, l), (prec, j, err)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c2_potentials_after_two_iterations(Plan, c2_ref, prec):
    xs, eps, l = c2_ref["xs"], C2["eps"], C2["l"]
    plan = Plan(xs, c2_ref["mus"], eps, precision=prec)
    plan.sinkhorn_step(2)
    for j in range(l):
        g = plan.get_potentials(j)
        ref = c2_ref["g2"][j]
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(g), fin)
        # errors of each product feed the next one; compare in units of eps
        err = float(np.max(np.abs(g[fin] - ref[fin]))) / eps
        assert err <= 20 * _tol(prec, ref / eps, xs, eps, l), (prec, j, err)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c2_stopping_residual_and_objective(Plan, c2_ref, prec):
    """The residual mmot_sinkhorn_step returns (Algorithm 1's stopping test,
    marginals 1..l-1) and the objective terms, both for the oracle's
    potentials after two iterations."""
    xs, mus, eps, l = c2_ref["xs"], c2_ref["mus"], C2["eps"], C2["l"]
    gs = c2_ref["g2"]
    plan = Plan(xs, mus, eps, precision=prec)
    for k in range(l):
        plan.set_potentials(k, gs[k])
    got = plan.sinkhorn_step(0, residual=True)
    ref, scale = _residual(xs, mus, gs, eps, range(l - 1))
    tol = 4 * _tol(prec, np.array([1.0]), xs, eps, l) * scale
    assert abs(got - ref) <= tol, (prec, got, ref, tol)
    obj = plan.objective()
    lnM, lnZ, W = oracle.allpass(xs, gs, eps)
    Z = math.exp(lnZ)
    otol = 4e-5 if prec == "fp32" else 1e-10
    assert abs(obj["mass"] - Z) <= otol * Z, (obj["mass"], Z)
    assert abs(obj["W"] - W) <= otol * abs(W), (obj["W"], W)
    marg = [np.exp(gs[k] / eps + lnM[k]) for k in range(l)]
    primal = sum(float(np.dot(gs[k], marg[k])) for k in range(l))
    pscale = sum(float(np.dot(np.abs(gs[k]), marg[k])) for k in range(l))
    assert abs(obj["primal"] - primal) <= otol * pscale, (obj["primal"], primal)
    res_all = sum(float(np.sum(np.abs(marg[k] - mus[k]))) for k in range(l))
    assert abs(obj["residual"] - res_all) <= otol * (res_all + Z), (obj["residual"], res_all)
    plan.close()


# ---- more tiles than one block of the carry scan ---------------------------

@pytest.fixture(scope="module")
def many_tiles_ref():
    l, N, eps = 3, 12_000_000, 2e-3
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=21)
    rng = np.random.default_rng(5)
    gs = [-eps * math.log(N) + 0.3 * eps * rng.standard_normal(N) for _ in range(l)]
    refs = {j: oracle.marginal_subset(xs, gs, eps, j) for j in (0, 2)}
    return dict(xs=xs, mus=mus, gs=gs, eps=eps, refs=refs)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_many_tiles(Plan, many_tiles_ref, prec):
    R = many_tiles_ref
    xs, eps = R["xs"], R["eps"]
    plan = Plan(xs, R["mus"], eps, precision=prec)
    assert plan.info()["tiles"] > 8192, plan.info()
    for k in range(3):
        plan.set_potentials(k, R["gs"][k])
    for j, ref in R["refs"].items():
        got = plan.marginal(j, "lnM")
        err = _lnM_err(got, ref)
        assert err <= _tol(prec, ref, xs, eps, 3), (prec, j, err)
    plan.close()


# ---- l = 8 at N = 2^16 -----------------------------------------------------

@pytest.fixture(scope="module")
def wide_ref():
    l, N, eps = 8, 1 << 16, 5e-3
    xs, mus = wl.sorted_uniform_dirichlet(l=l, N=N, instance=3)
    rng = np.random.default_rng(8)
    gs = [-eps * math.log(N) + 0.2 * eps * rng.standard_normal(N) for _ in range(l)]
    refs = {j: oracle.marginal_subset(xs, gs, eps, j) for j in (0, 3, 7)}
    return dict(xs=xs, mus=mus, gs=gs, eps=eps, refs=refs)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_l8_many_warp_tiles(Plan, wide_ref, prec):
    R = wide_ref
    xs, eps = R["xs"], R["eps"]
    plan = Plan(xs, R["mus"], eps, precision=prec)
    assert plan.info()["tiles"] >= 4096, plan.info()
    for k in range(8):
        plan.set_potentials(k, R["gs"][k])
    for j, ref in R["refs"].items():
        got = plan.marginal(j, "lnM")
        err = _lnM_err(got, ref)
        assert err <= _tol(prec, ref, xs, eps, 8), (prec, j, err)
    plan.close()


# ---- the stopping residual at other l --------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps", [(3, 20000, 1e-2), (5, 6000, 5e-3), (8, 1500, 2e-2)])
def test_stopping_residual(Plan, prec, l, N, eps):
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=60 + l)
    gs = _init_g(xs, eps)
    # three oracle iterations give potentials away from the start
    for _ in range(3):
        for j in range(l):
            gs[j] = oracle.potential_update(mus[j], oracle.marginal_subset(xs, gs, eps, j), eps)
    plan = Plan(xs, mus, eps, precision=prec)
    for k in range(l):
        plan.set_potentials(k, gs[k])
    got = plan.sinkhorn_step(0, residual=True)
    ref, scale = _residual(xs, mus, gs, eps, range(l - 1))
    tol = 4 * _tol(prec, np.array([1.0]), xs, eps, l) * scale
    assert abs(got - ref) <= tol, (prec, got, ref, tol)
    plan.close()


# ---- the FP32 path reaches the 1e-6 stopping tolerance -----------------------

@pytest.mark.parametrize("inst", [14, 8, 15, 58])
def test_fp32_solve_reaches_1e6_and_matches_fp64(Plan, inst):
    """Instances of the batched workload (l uniform in 3..8, N and eps
    log-uniform), one each of l = 3, 4, 5, 6: the FP32-scan solve stops at
    residual <= 1e-6 (Algorithm 1's stopping test), and its transport cost,
    mass and dual agree with the all-FP64 GPU solve at the same tolerance.
    (Instances at small eps that the FP64 solve itself does not bring to 1e-6
    within the budget are not used: there the two precisions stall together,
    their residuals agreeing to about 1e-5 relative.)"""
    l, N, eps = wl.batched_instance_params(64)[inst]
    xs, mus = wl.batched_instance(inst, l, N)
    out = {}
    for prec in ("fp32", "fp64"):
        plan = Plan(xs, mus, eps, precision=prec)
        out[prec] = plan.solve(1e-6, 20000)
        plan.close()
    for prec in ("fp32", "fp64"):
        assert out[prec]["converged"], (prec, out[prec])
        assert out[prec]["residual"] <= 1e-6, (prec, out[prec])
    a, b = out["fp32"], out["fp64"]
    assert abs(a["W"] - b["W"]) <= 1e-5 * abs(b["W"]), (a["W"], b["W"])
    assert abs(a["mass"] - b["mass"]) <= 1e-5, (a["mass"], b["mass"])
    assert abs(a["dual"] - b["dual"]) <= 1e-5 * abs(b["dual"]) + 1e-9, (a["dual"], b["dual"])
