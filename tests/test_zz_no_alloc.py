"""The allocation-free entry point mmot_marginal_noalloc (for callers that
cannot allocate device memory) against the CPU oracle.

Collected last on purpose.  Calls the C ABI directly, twice in a row on
different problems (the static working array keeps the previous call's
contents), and compares element by element with the oracle's subset chains
within the FP32 tolerance of the other GPU tests: 1e-5 on ln M, i.e. relative
1e-5 on M and on phi M.  Covers device and host inputs, the three output
kinds, and potentials written on a non-blocking stream right before the call
on that stream.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import _native
    return torch, _native.lib()


def _problem(l, N, eps, instance):
    from paper_2405_19246_gb300 import workloads as wl
    xs, mus = wl.sorted_uniform_lognormal(l=l, N=N, instance=instance)
    rng = np.random.default_rng(instance)
    gs = [-eps * np.log(N) + 0.5 * eps * rng.standard_normal(N) for _ in range(l)]
    return xs, gs


def _check(kind, got, lnM, g, eps):
    if kind == 2:
        err = float(np.max(np.abs(got - lnM)))
    elif kind == 0:
        err = float(np.max(np.abs(got / np.exp(lnM) - 1.0)))
    else:
        err = float(np.max(np.abs(got / np.exp(g / eps + lnM) - 1.0)))
    return err


def test_noalloc_matches_oracle_on_two_calls():
    torch, L = _setup()
    for call, (l, N, eps) in enumerate(((4, 5000, 5e-3), (3, 7000, 2e-2))):
        xs, gs = _problem(l, N, eps, 40 + call)
        dx = [torch.from_numpy(x).cuda() for x in xs]
        dg = [torch.from_numpy(g).cuda() for g in gs]
        Ns = (ctypes.c_int64 * l)(*[len(x) for x in xs])
        X = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dx])
        G = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dg])
        for k in range(l):
            lnM = oracle.marginal_subset(xs, gs, eps, k)
            for kind in (2, 0, 1):
                out = torch.full((len(xs[k]),), float("nan"), dtype=torch.float64, device="cuda")
                st = L.mmot_marginal_noalloc(l, Ns, X, G, eps, k, kind, out.data_ptr(), None)
                assert st == 0, L.mmot_last_error().decode()
                err = _check(kind, out.cpu().numpy(), lnM, gs[k], eps)
                assert err <= TOL, (call, k, kind, err)


def test_noalloc_host_inputs():
    torch, L = _setup()
    l, N, eps = 5, 3000, 1e-2
    xs, gs = _problem(l, N, eps, 47)
    Ns = (ctypes.c_int64 * l)(*[len(x) for x in xs])
    X = (ctypes.c_void_p * l)(*[x.ctypes.data for x in xs])
    G = (ctypes.c_void_p * l)(*[g.ctypes.data for g in gs])
    for k in (0, 4):
        lnM = oracle.marginal_subset(xs, gs, eps, k)
        out = torch.empty(N, dtype=torch.float64, device="cuda")
        st = L.mmot_marginal_noalloc(l, Ns, X, G, eps, k, 2, out.data_ptr(), None)
        assert st == 0, L.mmot_last_error().decode()
        assert _check(2, out.cpu().numpy(), lnM, gs[k], eps) <= TOL


def test_noalloc_reads_in_stream_order():
    """Potentials written on a non-blocking stream just before the call, on
    that same stream: the call must see the new values."""
    torch, L = _setup()
    l, N, eps = 4, 6000, 5e-3
    xs, gs = _problem(l, N, eps, 48)
    dx = [torch.from_numpy(x).cuda() for x in xs]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        host = [torch.from_numpy(g).pin_memory() for g in gs]
        dg = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in range(l)]
        for d, h in zip(dg, host):
            d.copy_(h, non_blocking=True)
            d.mul_(1.0)
        out = torch.empty(N, dtype=torch.float64, device="cuda")
        Ns = (ctypes.c_int64 * l)(*[N] * l)
        X = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dx])
        G = (ctypes.c_void_p * l)(*[t.data_ptr() for t in dg])
        st = L.mmot_marginal_noalloc(l, Ns, X, G, eps, 1, 2, out.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    assert st == 0, L.mmot_last_error().decode()
    s.synchronize()
    lnM = oracle.marginal_subset(xs, gs, eps, 1)
    assert _check(2, out.cpu().numpy(), lnM, gs[1], eps) <= TOL


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch, L = _setup()
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
