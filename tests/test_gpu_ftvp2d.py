"""The two-dimensional product (Sec. 4.1, Algorithm 6: FTVP_2d) on the GPU.

Against the oracle's dense definition (``oracle.brute.ftvp2d_dense``) on small
grids, element by element at 1e-13 relative (FP64, positive sums); at larger
grids against the separable closed form for rank-one inputs, whose factors
come from the literal one-dimensional Algorithm 2 of the C oracle.  Three
two-dimensional Sinkhorn updates (the update of Sec. 4.1 with the GPU
product) against the same updates with the dense product.
"""
import numpy as np
import pytest

import oracle
from oracle import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_19246_gb300 import api as a
    return a


@pytest.mark.parametrize("N,M,l1,l2", [(1, 1, 0.5, 0.5), (6, 5, 0.6, 0.8), (12, 9, 0.9, 0.3), (16, 16, 0.97, 0.97),
                                       (3, 20, 0.0, 0.7)])
def test_ftvp2d_matches_dense(api, N, M, l1, l2):
    rng = np.random.default_rng(N * 100 + M)
    phi = rng.random((N, M)) + 0.01
    psi = rng.random((N, M)) + 0.01
    got = api.ftvp2d(phi, psi, l1, l2)
    ref = brute.ftvp2d_dense(phi, psi, l1, l2)
    assert np.max(np.abs(got - ref) / ref) < 1e-13


def test_ftvp2d_rank_one_at_size(api):
    rng = np.random.default_rng(7)
    N, M = 300, 257
    a, b, c, d = rng.random(N), rng.random(N), rng.random(M), rng.random(M)
    got = api.ftvp2d(np.outer(a, c), np.outer(b, d), 0.95, 0.9)
    ref = np.outer(oracle.ftvp1(a, b, 0.95), oracle.ftvp1(c, d, 0.9))
    assert np.max(np.abs(got - ref) / ref) < 1e-12


def test_ftvp2d_sinkhorn_updates(api):
    """phi <- u / (K x psi x varphi) and so on (Sec. 4.1 updates), three
    rounds, with the GPU product and with the dense one."""
    rng = np.random.default_rng(9)
    N, M, l1, l2 = 8, 7, 0.7, 0.75
    u, v, w = (rng.random((N, M)) + 0.1 for _ in range(3))
    u, v, w = u / u.sum(), v / v.sum(), w / w.sum()

    def run(prod):
        phi = np.full((N, M), 1.0 / (N * M))
        psi, vphi = phi.copy(), phi.copy()
        for _ in range(3):
            phi = u / prod(psi, vphi)
            psi = v / prod(phi, vphi)
            vphi = w / prod(phi, psi)
        return phi, psi, vphi

    g = run(lambda a, b: api.ftvp2d(a, b, l1, l2))
    r = run(lambda a, b: brute.ftvp2d_dense(a, b, l1, l2))
    for x, y in zip(g, r):
        assert np.max(np.abs(x - y) / y) < 1e-12


def test_ftvp2d_rejects_bad_arguments(api):
    from paper_2405_19246_gb300 import _native as nat
    with pytest.raises(nat.MmotError):
        api.ftvp2d(np.ones((3, 3)), np.ones((3, 3)), 1.0, 0.5)
    with pytest.raises(ValueError):
        api.ftvp2d(np.ones((3, 3)), np.ones((3, 2)), 0.5, 0.5)
