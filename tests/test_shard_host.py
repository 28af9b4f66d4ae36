"""Shards of one instance, host side (no GPU): the cut into ranges of the
merged order and the exchange of transfer operators, with the per-range
operators and products taken from the brute-force definition in
``oracle.brute`` (sums over placements, the cost written as a sum over gaps).

Pinned by the dense tensor definition of M_j (Sec. 4.2, Eq. Jk k margin):
the states entering each range from the exchange, combined with the range's
own points, must give the dense M_j at every point, to rounding.  The
two-rank test runs the exchange as one all-gather over gloo ranks, one range
per rank (the multi-process path of ``shard.exchange_distributed``).
"""
import os
import socket

import numpy as np
import pytest

from oracle import brute
from paper_2405_19246_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _problem(l, n, eps, seed):
    rng = np.random.default_rng(seed)
    xs = [np.sort(rng.random(n)) for _ in range(l)]
    # a shared point between two marginals: ties across a cut are ordered by marginal
    xs[1][1] = xs[0][2]
    xs[1] = np.sort(xs[1])
    gs = [0.2 * rng.standard_normal(n) - eps * np.log(n) for _ in range(l)]
    return xs, gs


def _ranges(T, P):
    cuts = [(T * q) // P for q in range(P + 1)]
    return [(cuts[q], cuts[q + 1]) for q in range(P)]


def _range_ops(xs, gs, eps, j, lo, hi, X):
    e = (X[lo], X[hi - 1])
    return np.stack([brute.range_operator(xs, gs, eps, j, lo, hi, *e),
                     brute.range_operator(xs, gs, eps, j, lo, hi, *e, backward=True)]), e


@pytest.mark.parametrize("l,n,P", [(2, 5, 2), (3, 5, 3), (4, 4, 2), (4, 4, 4)])
def test_exchange_gives_dense_marginals(l, n, P):
    eps = 0.25
    xs, gs = _problem(l, n, eps, 10 + l + P)
    X, _, _ = brute.merged_order(xs)
    rg = _ranges(len(X), P)
    for j in range(l):
        ops, ends = zip(*[_range_ops(xs, gs, eps, j, lo, hi, X) for lo, hi in rg])
        lnF, lnG = shard.exchange(list(ops), list(ends), eps, l)
        got = np.concatenate([brute.ln_marginal_in_range(xs, gs, eps, j, lo, hi, lnF[q], lnG[q], *ends[q])
                              for q, (lo, hi) in enumerate(rg)])
        ref = brute.ln_marginal_product(xs, gs, eps, j)
        assert np.max(np.abs(got - ref)) <= 1e-12, (j, got, ref)
        # the first shard receives only the empty state from the left, the last from the right
        assert lnF[0][0] == 0.0 and np.all(np.isneginf(lnF[0][1:]))
        assert lnG[-1][0] == 0.0 and np.all(np.isneginf(lnG[-1][1:]))


def test_range_operator_diagonal_is_the_decay():
    l, eps = 3, 0.5
    xs, gs = _problem(l, 4, eps, 3)
    X, _, _ = brute.merged_order(xs)
    op = brute.range_operator(xs, gs, eps, 0, 2, 7, X[2], X[6])
    for s in range(l):
        assert op[s, 0] == pytest.approx(-s * (l - s) * (X[6] - X[2]) / eps, abs=1e-15)
    assert np.all(np.isneginf(op[2, 1:]))   # level l - 1 picks up nothing


def test_split_partitions_the_merged_order():
    rng = np.random.default_rng(4)
    l = 3
    xs = [np.sort(rng.random(50)) for _ in range(l)]
    mus = [np.full(50, 1 / 50) for _ in range(l)]
    parts = shard.split(xs, mus, 4)
    for k in range(l):
        assert np.array_equal(np.concatenate([p[0][k] for p in parts]), xs[k])
        assert np.array_equal(np.concatenate([p[1][k] for p in parts]), mus[k])
    ends = [shard.range_ends(p[0]) for p in parts]
    for a, b in zip(ends, ends[1:]):
        assert a[0] <= a[1] <= b[0] <= b[1]
    sizes = [sum(len(x) for x in p[0]) for p in parts]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError, match="no point of marginal"):
        shard.split([np.array([0.0, 0.1]), np.array([0.9, 1.0])], [np.full(2, 0.5)] * 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import brute as br
    from paper_2405_19246_gb300 import shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    l, eps = 4, 0.25
    xs, gs = _problem(l, 5, eps, 77)
    X, _, _ = br.merged_order(xs)
    lo, hi = _ranges(len(X), world)[rank]
    res = {}
    for j in range(l):
        ops, ends = _range_ops(xs, gs, eps, j, lo, hi, X)
        lnF, lnG = sh.exchange_distributed(ops, ends, eps, l)
        res[j] = br.ln_marginal_in_range(xs, gs, eps, j, lo, hi, lnF, lnG, *ends)
    out[rank] = res
    dist.destroy_process_group()


def test_exchange_on_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    l, eps = 4, 0.25
    xs, gs = _problem(l, 5, eps, 77)
    for j in range(l):
        got = np.concatenate([res[0][j], res[1][j]])
        ref = brute.ln_marginal_product(xs, gs, eps, j)
        assert np.max(np.abs(got - ref)) <= 1e-12, j
