"""The allocation-free entry point mmot_marginal_noalloc, for callers that
cannot allocate device memory, against the plan-based mmot_marginal.

Collected last on purpose.  Calls the C ABI directly, twice in a row on
different problems (the static working array keeps the previous call's
contents), and compares ln M_k element by element within the FP32 tolerance
of the other GPU tests (1e-5 on ln M, i.e. relative 1e-5 on M).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_plan_marginal_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import _native
    from paper_2405_19246_gb300 import workloads as wl
    from paper_2405_19246_gb300.api import Plan

    L = _native.lib()
    for call, (l, N, eps) in enumerate(((4, 5000, 5e-3), (3, 7000, 2e-2))):
        xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=40 + call)
        plan = Plan(xs, mus, eps, precision="fp32")
        plan.sinkhorn_step(2)
        gs = [plan.get_potentials(k) for k in range(l)]
        dx = [torch.from_numpy(x).cuda() for x in xs]
        dg = [torch.from_numpy(g).cuda() for g in gs]
        Ns = (ctypes.c_int64 * l)(*[len(x) for x in xs])
        X = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dx])
        G = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dg])
        for k in range(l):
            ref = plan.marginal(k, "lnM")
            out = torch.full((len(xs[k]),), float("nan"), dtype=torch.float64, device="cuda")
            st = L.mmot_marginal_noalloc(l, Ns, X, G, eps, k, 2, out.data_ptr(), None)
            assert st == 0, L.mmot_last_error().decode()
            got = out.cpu().numpy()
            err = float(np.max(np.abs(got - ref)))
            assert err <= TOL, (call, k, err)
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import _native
    L = _native.lib()
    l, N = 2, 300000   # 600000 points > 2^19
    xs = [torch.linspace(0, 1, N, dtype=torch.float64, device="cuda") for _ in range(l)]
    gs = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(l)]
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    Ns = (ctypes.c_int64 * l)(N, N)
    X = (ctypes.c_void_p * l)(*[t.data_ptr() for t in xs])
    G = (ctypes.c_void_p * l)(*[t.data_ptr() for t in gs])
    st = L.mmot_marginal_noalloc(l, Ns, X, G, 0.1, 0, 2, out.data_ptr(), None)
    assert st == 8   # MMOT_ERR_RANGE
    assert b"static scratch limit" in L.mmot_last_error()
