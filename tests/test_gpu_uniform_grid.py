"""Uniform-grid specialisation: every marginal on one grid x_i = x_0 + i h,
the setting of Sec. 3 (Algorithms 2, 3 and 5 take a constant lambda = e^{-h/eps}
per grid step).  The plan detects it and the tile kernels then form each
point's position factor e^{pos} (a table of e^{d h/eps} by grid steps d) and
its marginal (merged index mod l) instead of reading them from the stream.

Parity against the oracle element by element (1e-5 on ln M for the FP32
path, 1e-12 for FP64, scaled by the magnitude of the log values), on grids
whose tiles start in the middle of a grid point (the tile length is not a
multiple of l), and against the general path on the same problem with the
grid perturbed off uniformity.
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


def _tol(prec, ref, eps, xmax, l):
    fin = ref[np.isfinite(ref)]
    t = TOL[prec] * max(1.0, 1e-2 * float(np.max(np.abs(fin))))
    if prec == "fp64":
        t += 8 * 1.1102230246251565e-16 * (l // 2) * ((l + 1) // 2) * xmax / eps
    return t


def _problem(l, N, eps, seed, perturb=0.0):
    rng = np.random.default_rng(seed)
    x = np.linspace(-1.0, 2.0, N)
    if perturb:
        x = x + perturb * (x[1] - x[0]) * np.sin(np.arange(N))
    xs = [x.copy() for _ in range(l)]
    mus = []
    for _ in range(l):
        w = rng.random(N) + 0.05
        mus.append(w / w.sum())
    gs = [-eps * math.log(N) + 0.3 * eps * rng.standard_normal(N) for _ in range(l)]
    return xs, mus, gs


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("l,N,eps", [(3, 20000, 2e-3), (4, 9000, 5e-3), (5, 4000, 1e-2), (2, 30000, 1e-3)])
def test_uniform_grid_products_match_oracle(Plan, prec, l, N, eps):
    xs, mus, gs = _problem(l, N, eps, 300 + l)
    p = Plan(xs, mus, eps, precision=prec)
    info = p.info()
    assert info["uniform_grid"] == 1, info
    assert info["tiles"] >= 4, info
    for k in range(l):
        p.set_potentials(k, gs[k])
    for j in range(l):
        ref = oracle.marginal_subset(xs, gs, eps, j)
        got = p.marginal(j, "lnM")
        err = float(np.max(np.abs(got - ref)))
        assert err <= _tol(prec, ref, eps, 2.0, l), (prec, l, j, err)
    p.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_uniform_grid_iterations_match_general_path(Plan, prec):
    """Five Sinkhorn iterations on a uniform grid and on the same grid moved
    off uniformity by 1e-7 of a step (general path): the plans agree to the
    perturbation's effect, and the uniform one matches the oracle's driver."""
    l, N, eps = 3, 6000, 5e-3
    xs, mus, _ = _problem(l, N, eps, 77)
    xs2, _, _ = _problem(l, N, eps, 77, perturb=1e-7)
    a = Plan(xs, mus, eps, precision=prec)
    b = Plan(xs2, mus, eps, precision=prec)
    assert a.info()["uniform_grid"] == 1 and b.info()["uniform_grid"] == 0
    ra = a.sinkhorn_step(5, residual=True)
    rb = b.sinkhorn_step(5, residual=True)
    ref = oracle.sinkhorn(xs, mus, eps, 0.0, 5)
    for k in range(l):
        ga, gb = a.get_potentials(k), b.get_potentials(k)
        scale = 1e-4 if prec == "fp32" else 1e-9
        assert float(np.max(np.abs(ga - ref["g"][k]))) <= scale * eps * 50, k
        assert float(np.max(np.abs(ga - gb))) <= scale * eps * 50 + 1e-6 * eps, k
    assert abs(ra - rb) <= 1e-3 * max(ra, 1e-6)
    a.close()
    b.close()


def test_grid_workloads_use_the_uniform_path(Plan):
    for xs, mus in (wl.uniform_grid_mixture(l=3, N=1000), wl.paper_random_1d(80), wl.paper_ricker(100)):
        p = Plan(xs, mus, 1e-2)
        assert p.info()["uniform_grid"] == 1
        p.close()
    xs, mus = wl.sorted_uniform_lognormal(l=3, N=1000, instance=1)
    p = Plan(xs, mus, 1e-2)
    assert p.info()["uniform_grid"] == 0
    p.close()
