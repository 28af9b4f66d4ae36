"""Pins for the CPU oracle against facts that do not come from the oracle itself:
the dense definition (brute force), closed forms, limits, invariants and
symmetries of the l-marginal product with L1 cost (Sec. 3 and Sec. 4.2)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_2405_19246_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _rand_potentials(xs, seed, scale=0.05, neg_inf_every=0):
    rng = np.random.default_rng(seed)
    gs = [rng.normal(size=len(x)) * scale for x in xs]
    if neg_inf_every:
        for k in range(0, len(gs), neg_inf_every):
            gs[k][len(gs[k]) // 2] = -np.inf
    return gs


CASES = [
    (2, (6, 5), False, False),
    (3, (5, 7, 4), False, False),
    (3, (6, 6, 6), True, False),
    (4, (5, 4, 6, 3), False, True),
    (4, (6, 6, 6, 6), True, True),
    (5, (4, 3, 5, 4, 3), True, False),
]


@pytest.mark.parametrize("l,Ns,ties,zeros", CASES)
def test_subset_and_classes_match_dense_definition(l, Ns, ties, zeros):
    xs, _ = wl.random_small(l, Ns, seed=10 * l + ties, ties=ties)
    eps = 0.06
    gs = _rand_potentials(xs, 3 + l, neg_inf_every=2 if zeros else 0)
    for j in range(l):
        ref = brute.ln_marginal_product(xs, gs, eps, j)
        sub = oracle.marginal_subset(xs, gs, eps, j)
        cls = oracle.marginal_classes(xs, gs, eps, j)
        np.testing.assert_allclose(sub, ref, rtol=0, atol=1e-12)
        np.testing.assert_allclose(cls, ref, rtol=0, atol=1e-12)


def test_sampled_subset_equals_full():
    xs, _ = wl.random_small(4, (30, 20, 25, 15), seed=5)
    gs = _rand_potentials(xs, 9)
    full = oracle.marginal_subset(xs, gs, 0.03, 2)
    want = [0, 3, 7, 24]
    part = oracle.marginal_subset(xs, gs, 0.03, 2, want=want)
    np.testing.assert_array_equal(part, full[want])


@pytest.mark.parametrize("l,Ns,ties,zeros", CASES)
def test_allpass_marginals_mass_and_cost(l, Ns, ties, zeros):
    xs, _ = wl.random_small(l, Ns, seed=7 * l, ties=ties)
    eps = 0.08
    gs = _rand_potentials(xs, l, neg_inf_every=3 if zeros else 0)
    lnMs, lnZ, W = oracle.allpass(xs, gs, eps)
    for j in range(l):
        np.testing.assert_allclose(lnMs[j], brute.ln_marginal_product(xs, gs, eps, j), atol=1e-12)
    T = brute.plan(xs, gs, eps)
    assert math.isclose(math.exp(lnZ), T.sum(), rel_tol=1e-12)
    assert math.isclose(W, brute.transport_cost(xs, gs, eps), rel_tol=1e-12)


def test_l2_geometric_closed_form():
    N, h, eps = 40, 0.1, 0.07
    lam = math.exp(-h / eps)
    x = np.arange(N) * h
    xs = [x, x.copy()]
    gs = [np.zeros(N), np.zeros(N)]
    i = np.arange(N)
    ref = (1 - lam ** (i + 1)) / (1 - lam) + lam * (1 - lam ** (N - 1 - i)) / (1 - lam)
    for j in range(2):
        got = np.exp(oracle.marginal_subset(xs, gs, eps, j))
        np.testing.assert_allclose(got, ref, rtol=1e-13)


def test_l3_interior_closed_form_golden():
    g = json.load(open(GOLDEN))["l3_interior_all_ones"]
    lam = g["lambda"]
    assert math.isclose(1 + 6 * lam ** 2 / (1 - lam ** 2) ** 2, g["value"], rel_tol=1e-15)
    N = 201
    eps = -1.0 / math.log(lam)        # h = 1, lambda = exp(-h/eps)
    x = np.arange(N, dtype=np.float64)
    xs = [x, x.copy(), x.copy()]
    gs = [np.zeros(N)] * 3
    for j in range(3):
        got = math.exp(oracle.marginal_subset(xs, gs, eps, j)[N // 2])
        assert math.isclose(got, g["value"], rel_tol=1e-13)
    # Algorithm 2 on the same grid
    out = oracle.ftvp1(np.ones(N), np.ones(N), lam)
    assert math.isclose(out[N // 2], g["value"], rel_tol=1e-13)


def test_large_eps_limit_is_product_of_sums():
    xs, _ = wl.random_small(4, (7, 5, 6, 4), seed=2)
    gs = _rand_potentials(xs, 4, scale=1.0)
    eps = 1e9
    # scale potentials with eps so that phi stays O(1)
    gsc = [g * eps for g in gs]
    for j in range(4):
        got = np.exp(oracle.marginal_subset(xs, gsc, eps, j))
        ref = np.prod([np.exp(gs[m]).sum() for m in range(4) if m != j])
        np.testing.assert_allclose(got, ref, rtol=1e-7)


def test_mass_is_the_same_for_every_marginal():
    xs, _ = wl.random_small(5, (9, 8, 7, 10, 6), seed=1)
    gs = _rand_potentials(xs, 1, scale=0.3)
    eps = 0.05
    _, lnZ, _ = oracle.allpass(xs, gs, eps)
    for j in range(5):
        lnM = oracle.marginal_subset(xs, gs, eps, j)
        Z = np.sum(np.exp(gs[j] / eps + lnM))
        assert math.isclose(Z, math.exp(lnZ), rel_tol=1e-12)


def test_reflection_translation_and_scaling_symmetry():
    xs, _ = wl.random_small(4, (8, 6, 7, 5), seed=4)
    gs = _rand_potentials(xs, 8, scale=0.1)
    eps = 0.04
    base = [oracle.marginal_subset(xs, gs, eps, j) for j in range(4)]
    # reflection x -> -x reverses every support
    xr = [(-x)[::-1].copy() for x in xs]
    gr = [g[::-1].copy() for g in gs]
    # translation
    xt = [x + 3.75 for x in xs]
    # scaling of x and eps together
    a = 2.5
    xsc = [a * x for x in xs]
    for j in range(4):
        np.testing.assert_allclose(oracle.marginal_subset(xr, gr, eps, j)[::-1], base[j], atol=1e-12)
        np.testing.assert_allclose(oracle.marginal_subset(xt, gs, eps, j), base[j], atol=1e-12)
        # phi = exp(g/eps) is unchanged when g scales with eps
        np.testing.assert_allclose(oracle.marginal_subset(xsc, [a * g for g in gs], a * eps, j),
                                   base[j], atol=1e-12)


def test_ftvp1_and_ftvp2_match_dense_definition():
    N = 17
    h = 1.0 / (N - 1)
    eps = 0.05
    lam = math.exp(-h / eps)
    rng = np.random.default_rng(0)
    phi, psi = rng.random(N) + 0.1, rng.random(N) + 0.1
    x = np.linspace(0, 1, N)
    xs = [x, x, x]
    C = brute.cost_tensor(xs)
    K = np.exp(-C / eps)
    ref1 = np.einsum("ijk,i,j->k", K, phi, psi)
    ref2 = np.einsum("ijk,i,j->k", C * K, phi, psi)
    np.testing.assert_allclose(oracle.ftvp1(phi, psi, lam), ref1, rtol=1e-13)
    np.testing.assert_allclose(oracle.ftvp2(phi, psi, lam, h), ref2, rtol=1e-12)


def test_fs3_matches_general_driver_and_dense_plan():
    """Algorithm 4 (literal l = 3) vs the general log-domain driver, and the
    fast plan vs dense Sinkhorn as in Table 'table1' (Sec. 5.1)."""
    g = json.load(open(GOLDEN))["table3_fast_vs_dense"]
    for N in (10, 20):
        xs, mus = wl.paper_random_1d(N)
        eps, iters = 0.1, 100
        h = 1.0 / (N - 1)
        r = oracle.fs3(*mus, h=h, eps=eps, tol=0.0, itr_max=iters)
        s = oracle.sinkhorn(xs, mus, eps, 0.0, iters)
        assert r["iters"] == iters == s["iters"]
        assert math.isclose(r["W"], s["W"], rel_tol=1e-12)
        gf = [eps * np.log(r["phi"]), eps * np.log(r["psi"]), eps * np.log(r["varphi"])]
        for a, b in zip(gf, s["g"]):
            np.testing.assert_allclose(a, b, atol=1e-12)
        gd = brute.sinkhorn_dense(xs, mus, eps, iters)
        P_fast = brute.plan(xs, gf, eps)
        P_dense = brute.plan(xs, gd, eps)
        assert np.linalg.norm((P_fast - P_dense).ravel()) < 1e-14
        assert max(g["frobenius_plan_difference"]) < 1e-14


def test_sinkhorn_matches_dense_l4_n20():
    """Brute-force dense check at N = 20, l = 4 on the grid-mixture law."""
    xs, mus = wl.uniform_grid_mixture(l=4, N=20)
    eps = 1e-1
    s = oracle.sinkhorn(xs, mus, eps, 0.0, 3)
    gd = brute.sinkhorn_dense(xs, mus, eps, 3)
    for a, b in zip(s["g"], gd):
        np.testing.assert_allclose(a, b, atol=1e-12)
    assert math.isclose(s["W"], brute.transport_cost(xs, s["g"], eps), rel_tol=1e-12)


def test_sinkhorn_block_update_invariants():
    """After updating marginal j it is matched exactly; the dual objective
    sum <g, mu> + eps - eps Z never decreases over block updates (exact block
    coordinate ascent); the plan is positive."""
    xs, mus = wl.random_small(4, (9, 7, 8, 6), seed=3, zeros=True)
    eps = 0.05
    gs = [np.full(len(x), -eps * math.log(len(x))) for x in xs]

    def dual(gs):
        _, lnZ, _ = oracle.allpass(xs, gs, eps)
        return sum(float(np.sum(np.where(np.isfinite(g), g, 0.0) * m)) for g, m in zip(gs, mus)) \
            + eps - eps * math.exp(lnZ)

    prev = dual(gs)
    for it in range(6):
        for j in range(4):
            lnM = oracle.marginal_subset(xs, gs, eps, j)
            gs[j] = oracle.potential_update(mus[j], lnM, eps)
            lnM2 = oracle.marginal_subset(xs, gs, eps, j)
            marg = np.where(np.isfinite(gs[j]), np.exp(gs[j] / eps + lnM2), 0.0)
            np.testing.assert_allclose(marg, mus[j], rtol=1e-12, atol=1e-300)
            d = dual(gs)
            assert d >= prev - 1e-13
            prev = d
    assert np.all(brute.plan(xs, gs, eps) >= 0)


def test_sinkhorn_converges_gap_closes():
    xs, mus = wl.random_small(3, (12, 10, 11), seed=8)
    eps = 0.1
    s = oracle.sinkhorn(xs, mus, eps, 1e-10, 5000)
    assert s["res"] <= 1e-10
    assert abs(s["primal"] - s["dual"]) < 1e-9
    assert math.isclose(s["mass"], 1.0, rel_tol=1e-9)
    T = brute.plan(xs, s["g"], eps)
    for k in range(3):
        axes = tuple(a for a in range(3) if a != k)
        np.testing.assert_allclose(T.sum(axis=axes), mus[k], atol=1e-10)


def test_ricker_fs3_vs_general():
    xs, mus = wl.paper_ricker(40)
    h = 4.0 / 39
    r = oracle.fs3(*mus, h=h, eps=0.1, tol=0.0, itr_max=50)
    s = oracle.sinkhorn(xs, mus, 0.1, 0.0, 50)
    assert math.isclose(r["W"], s["W"], rel_tol=1e-12)


def test_grid_mixture_c1_fs3_vs_general():
    """The l = 3, N = 1000, eps = 1e-2, 200-iteration grid-mixture workload by the
    literal Algorithm 4 and by the general subset-chain driver."""
    xs, mus = wl.uniform_grid_mixture(l=3, N=1000)
    eps, iters = 1e-2, 200
    r = oracle.fs3(*mus, h=1.0 / 999, eps=eps, tol=0.0, itr_max=iters)
    s = oracle.sinkhorn(xs, mus, eps, 0.0, iters)
    assert math.isclose(r["W"], s["W"], rel_tol=1e-10)
    gf = [eps * np.log(r["phi"]), eps * np.log(r["psi"]), eps * np.log(r["varphi"])]
    for a, b in zip(gf, s["g"]):
        np.testing.assert_allclose(a, b, atol=1e-9)


def test_unsorted_support_rejected():
    with pytest.raises(ValueError):
        oracle.merge([np.array([0.0, 1.0]), np.array([0.5, 0.2])])


def test_merge_tie_rule():
    """Equal coordinates are ordered by marginal index (the tie rule of D_p)."""
    mid, loc = oracle.merge([np.array([0.0, 1.0]), np.array([0.0, 1.0]), np.array([0.5])])
    assert list(mid) == [0, 1, 2, 0, 1]
    assert list(loc) == [0, 0, 0, 1, 1]


# ---- the two-dimensional product (Sec. 4.1) -----------------------------------

def test_ftvp2d_dense_separates_for_rank_one_inputs():
    """For phi = a c^T and psi = b d^T the separable kernel gives
    J = FTVP1(a, b; lam1) FTVP1(c, d; lam2)^T, each factor from the literal
    Algorithm 2 of the C oracle (an independent code path)."""
    from oracle import brute
    rng = np.random.default_rng(12)
    a, b = rng.random(6), rng.random(6)
    c, d = rng.random(5), rng.random(5)
    J = brute.ftvp2d_dense(np.outer(a, c), np.outer(b, d), 0.6, 0.8)
    ref = np.outer(oracle.ftvp1(a, b, 0.6), oracle.ftvp1(c, d, 0.8))
    assert np.max(np.abs(J - ref) / ref) < 1e-13


def test_ftvp2d_dense_with_one_column_is_the_1d_product():
    from oracle import brute
    rng = np.random.default_rng(13)
    a, b = rng.random(9), rng.random(9)
    J = brute.ftvp2d_dense(a[:, None], b[:, None], 0.5, 0.9)
    assert np.max(np.abs(J[:, 0] - oracle.ftvp1(a, b, 0.5)) / J[:, 0]) < 1e-13
