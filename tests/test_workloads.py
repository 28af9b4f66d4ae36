"""The seeded input generators: deterministic, with the shapes and value
distributions of the configurations they stand for (no method arithmetic)."""
import math

import numpy as np

from paper_2405_19246_gb300 import workloads as wl


def _check_instance(xs, mus, l, N):
    assert len(xs) == l and len(mus) == l
    for x, m in zip(xs, mus):
        assert len(x) == N and len(m) == N
        assert np.all(np.diff(x) >= 0)
        assert np.all(m >= 0)
        assert abs(m.sum() - 1.0) <= 1e-12


def test_generators_are_deterministic_and_well_formed():
    a = wl.sorted_uniform_lognormal(l=4, N=1000, instance=3)
    b = wl.sorted_uniform_lognormal(l=4, N=1000, instance=3)
    c = wl.sorted_uniform_lognormal(l=4, N=1000, instance=4)
    for k in range(4):
        np.testing.assert_array_equal(a[0][k], b[0][k])
        np.testing.assert_array_equal(a[1][k], b[1][k])
        assert not np.array_equal(a[0][k], c[0][k])
    _check_instance(*a, 4, 1000)
    _check_instance(*wl.sorted_uniform_dirichlet(l=8, N=500), 8, 500)
    xs, mus = wl.uniform_grid_mixture(l=3, N=1000)
    _check_instance(xs, mus, 3, 1000)
    np.testing.assert_allclose(np.diff(xs[0]), 1.0 / 999, rtol=1e-9)


def test_supports_lie_in_the_unit_interval_and_weights_follow_their_laws():
    xs, mus = wl.sorted_uniform_lognormal(l=2, N=200000, instance=1)
    x = xs[0]
    assert 0.0 <= x[0] and x[-1] < 1.0
    # sorted U[0,1]: the empirical CDF is uniform
    assert np.max(np.abs(np.arange(1, len(x) + 1) / len(x) - x)) < 0.01
    # LogNormal(0,1) weights: the logs of the unnormalised weights have sd 1
    lm = np.log(mus[0])
    assert abs(np.std(lm) - 1.0) < 0.01
    # Dirichlet(1) weights: normalised Exp(1), coefficient of variation 1
    _, mus = wl.sorted_uniform_dirichlet(l=1, N=200000)
    m = mus[0]
    assert abs(np.std(m) / np.mean(m) - 1.0) < 0.02


def test_batched_parameters_follow_the_configured_ranges():
    p = wl.batched_instance_params(4096)
    ls = np.array([q[0] for q in p])
    Ns = np.array([q[1] for q in p])
    eps = np.array([q[2] for q in p])
    assert set(ls.tolist()) == set(range(3, 9))
    assert Ns.min() >= 64 and Ns.max() <= 65536
    assert eps.min() >= 1e-3 and eps.max() <= 1e-1
    # log-uniform: the logs are spread evenly over the range
    u = (np.log(Ns) - math.log(64)) / (math.log(65536) - math.log(64))
    assert abs(np.mean(u) - 0.5) < 0.02
    v = (np.log(eps) - math.log(1e-3)) / (math.log(1e-1) - math.log(1e-3))
    assert abs(np.mean(v) - 0.5) < 0.02
    assert p == wl.batched_instance_params(4096)
    xs, mus = wl.batched_instance(7, *p[7][:2])
    _check_instance(xs, mus, p[7][0], p[7][1])


def test_paper_workloads():
    xs, mus = wl.paper_random_1d(300)
    _check_instance(xs, mus, 3, 300)
    xs, mus = wl.paper_ricker(256)
    assert len(xs) == 3
    for m in mus:
        assert np.all(m > 0) and abs(m.sum() - 1.0) <= 1e-12
