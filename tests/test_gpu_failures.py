"""Failure paths, in forms that fault and hang no GPU.

* A bounded inter-tile wait that runs out: the test hook MMOT_OPT_TEST_HOLD
  keeps the first chunk of the carry scans from publishing its flags, so the
  waits of the later chunks reach their (short) poll limit; the call returns
  MMOT_ERR_TIMEOUT and the context stays usable for the next plan.  The
  products (carry scan for l <= 5, level scans for l >= 6) and, for l = 4,
  the objective sweeps are covered.
* A potential update that becomes infinite: every potential of one marginal
  set to -inf (zero scaling) makes the other products zero, so the update
  ln mu - ln M is +inf: MMOT_ERR_NONFINITE.
* The iteration cap: MMOT_ERR_NOT_CONVERGED with the result filled.
* A device-memory cap below what a plan needs: MMOT_ERR_OOM before any
  allocation crosses it, and the next creation without the cap succeeds.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2405_19246_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Plan():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300.api import Plan as P
    return P


@pytest.mark.parametrize("l,N", [(4, 60000), (7, 4000)])
def test_bounded_wait_times_out(Plan, l, N):
    from paper_2405_19246_gb300 import _native as nat
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=70 + l)
    eps = 1e-2
    plan = Plan(xs, mus, eps, precision="fp32")
    assert plan.info()["tiles"] > 64
    plan.set_option(nat.MMOT_OPT_SPIN_LIMIT, 2000)
    plan.set_option(nat.MMOT_OPT_TEST_HOLD, 1)
    with pytest.raises(nat.MmotError) as ei:
        plan.marginal(0, "lnM")
    assert ei.value.status == 5   # MMOT_ERR_TIMEOUT
    with pytest.raises(nat.MmotError) as ei:
        plan.sinkhorn_step(1)
    assert ei.value.status == 5
    if l <= 4:
        with pytest.raises(nat.MmotError) as ei:
            plan.objective()
        assert ei.value.status == 5
    # the hook off again: the same plan and a fresh one give correct products
    plan.set_option(nat.MMOT_OPT_TEST_HOLD, 0)
    plan.reset_potentials()
    gs = [np.full(len(x), -eps * math.log(len(x))) for x in xs]
    ref = oracle.marginal_subset(xs, gs, eps, 1)
    assert float(np.max(np.abs(plan.marginal(1, "lnM") - ref))) <= 1e-5
    plan.close()
    plan2 = Plan(xs, mus, eps, precision="fp32")
    assert float(np.max(np.abs(plan2.marginal(1, "lnM") - ref))) <= 1e-5
    plan2.close()


@pytest.mark.parametrize("l", [3, 6])
def test_infinite_potential_update_is_reported(Plan, l):
    from paper_2405_19246_gb300 import _native as nat
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=2000, instance=80 + l)
    plan = Plan(xs, mus, 2e-2, precision="fp32")
    plan.set_potentials(1, np.full(len(xs[1]), -np.inf))
    with pytest.raises(nat.MmotError) as ei:
        plan.sinkhorn_step(1)
    assert ei.value.status == 7   # MMOT_ERR_NONFINITE
    plan.close()


def test_iteration_cap_returns_not_converged_with_result(Plan):
    from paper_2405_19246_gb300 import _native as nat
    import ctypes
    xs, mus = wl.sorted_uniform_lognormal(l=4, N=3000, instance=90)
    plan = Plan(xs, mus, 1e-2, precision="fp32")
    res = nat.MmotResult()
    st = nat.lib().mmot_solve(plan._h, 1e-12, 2, ctypes.byref(res))
    assert st == 6   # MMOT_ERR_NOT_CONVERGED
    assert res.iters == 2
    assert res.residual > 1e-12 and math.isfinite(res.residual)
    assert math.isfinite(res.W) and res.W > 0 and res.mass > 0
    plan.close()


def test_memory_limit_gives_oom(Plan):
    from paper_2405_19246_gb300 import _native as nat
    xs, mus = wl.sorted_uniform_lognormal(l=4, N=5000, instance=91)
    L = nat.lib()
    used = ctypes.c_int64()
    plan = Plan(xs, mus, 1e-2, precision="fp32")
    need = plan.info()["device_bytes"]
    plan.close()
    assert need > 0
    # the cap counts what other live plans of this process hold as well
    assert L.mmot_memory_in_use(ctypes.byref(used)) == 0
    base = used.value
    try:
        assert L.mmot_set_memory_limit(base + need // 2) == 0
        with pytest.raises(nat.MmotError) as ei:
            Plan(xs, mus, 1e-2, precision="fp32")
        assert ei.value.status == 3   # MMOT_ERR_OOM
        assert L.mmot_memory_in_use(ctypes.byref(used)) == 0
        assert used.value == base   # the failed creation freed what it took
        assert L.mmot_set_memory_limit(base + need + (1 << 20)) == 0
        plan = Plan(xs, mus, 1e-2, precision="fp32")
        assert plan.info()["device_bytes"] == need
        plan.close()
    finally:
        L.mmot_set_memory_limit(0)


def test_set_potentials_rejects_nan_and_keeps_the_plan(Plan):
    """mmot_set_potentials checks its input on the device before it changes
    anything: a NaN or +inf is MMOT_ERR_INVALID_ARG and the plan keeps its
    potentials; host and device inputs then give the oracle's products."""
    import torch
    from paper_2405_19246_gb300 import _native as nat
    l, N, eps = 4, 3000, 1e-2
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=95)
    rng = np.random.default_rng(95)
    gs = [-eps * math.log(N) + 0.5 * eps * rng.standard_normal(N) for _ in range(l)]
    gs[2][::7] = -np.inf   # zero scalings are allowed
    plan = Plan(xs, mus, eps, precision="fp32")
    for k in range(l):
        if k % 2:
            plan.set_potentials(k, torch.from_numpy(gs[k]).cuda())
        else:
            plan.set_potentials(k, gs[k])
    before = [plan.get_potentials(k) for k in range(l)]
    for bad in (np.nan, np.inf):
        g = gs[1].copy()
        g[N // 2] = bad
        with pytest.raises(nat.MmotError) as ei:
            plan.set_potentials(1, g)
        assert ei.value.status == 1   # MMOT_ERR_INVALID_ARG
    for k in range(l):
        assert np.array_equal(plan.get_potentials(k), before[k])
    for j in range(l):
        ref = oracle.marginal_subset(xs, gs, eps, j)
        got = plan.marginal(j, "lnM")
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        assert float(np.max(np.abs(got[fin] - ref[fin]))) <= 1e-5, j
    plan.close()
