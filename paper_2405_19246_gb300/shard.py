"""One instance split into shards of the merged order (the host side of the
shard calls in ``include/mmot.h``).

A shard is a contiguous range of the merged order of all support points
(sorted by x, then marginal, then index).  Its plan holds every point of every
marginal in the range, so potentials never leave their shard.  For a product
of target k the only thing that crosses a cut is the vector of subset states
of Sec. 4.2 there (2^(l-1) forward states entering from the left, as many
backward states from the right).  The states leaving a range are linear in the
states entering it, through the shard's transfer operator (computed on the
device by ``mmot_shard_operator``); :func:`exchange` composes the operators of
all shards in order, with the decay exp(-w_s gap/eps) of a level-s state
(w_s = s(l - s), Sec. 4.2) across each gap between neighbours, and returns the
states entering every shard.  That is the whole exchange: at most
2 l 2^(l-1) numbers per shard and product, gathered from every shard (one
all-gather in a multi-process run, :func:`exchange_distributed`).

:class:`ShardedPlan` drives P shard plans on one GPU through Algorithm 1's
Gauss-Seidel iteration with this host exchange; a multi-GPU run puts one
shard per process and replaces the list of operators by the all-gather.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat
from .api import _PREC, _KIND

_NEG = -np.inf


def _popcounts(NS):
    return np.array([bin(T).count("1") for T in range(NS)], dtype=np.int64)


def split(xs, mus, n_shards):
    """Cut the merged order into n_shards contiguous ranges of about equal
    size.  Returns a list of (xs_q, mus_q) per shard (each a list of l numpy
    arrays: the points of marginal k inside the range, in their order).
    Raises ValueError if a range would hold no point of some marginal."""
    l = len(xs)
    xs = [np.asarray(x, dtype=np.float64) for x in xs]
    mus = [np.asarray(m, dtype=np.float64) for m in mus]
    allx = np.concatenate(xs)
    allk = np.concatenate([np.full(len(x), k) for k, x in enumerate(xs)])
    alli = np.concatenate([np.arange(len(x)) for x in xs])
    order = np.lexsort((alli, allk, allx))   # merged order: x, then marginal, then index
    T = len(order)
    if not 1 <= n_shards <= T:
        raise ValueError("n_shards = %d outside [1, %d]" % (n_shards, T))
    cuts = [(T * q) // n_shards for q in range(n_shards + 1)]
    # the merged position of every point, per marginal
    pos = np.empty(T, dtype=np.int64)
    pos[order] = np.arange(T)
    starts = np.cumsum([0] + [len(x) for x in xs])
    out = []
    for q in range(n_shards):
        xq, mq = [], []
        for k in range(l):
            pk = pos[starts[k]:starts[k + 1]]
            sel = (pk >= cuts[q]) & (pk < cuts[q + 1])
            if not sel.any():
                raise ValueError("shard %d holds no point of marginal %d" % (q, k))
            xq.append(np.ascontiguousarray(xs[k][sel]))
            mq.append(np.ascontiguousarray(mus[k][sel]))
        out.append((xq, mq))
    return out


def range_ends(xs_q):
    """x_L, x_R of a shard: its first and last point in the merged order."""
    return float(min(x[0] for x in xs_q)), float(max(x[-1] for x in xs_q))


def _apply(op, lnin, pc):
    """ln of the states leaving a range: out[T] = logsumexp over S inside T
    of lnin[S] + op[|S|][T \\ S] (op[s][0] the decay of level s)."""
    NS = len(lnin)
    out = np.full(NS, _NEG)
    for T in range(NS):
        terms = []
        S = T
        while True:
            if lnin[S] > _NEG and op[pc[S], T ^ S] > _NEG:
                terms.append(lnin[S] + op[pc[S], T ^ S])
            if S == 0:
                break
            S = (S - 1) & T
        if terms:
            m = max(terms)
            out[T] = m + np.log(np.sum(np.exp(np.array(terms) - m)))
    return out


def exchange(lnops, ends, eps, l):
    """States entering each shard for one target.

    lnops: per shard the [2, l, 2^(l-1)] array of ``mmot_shard_operator``
    (shard order); ends: per shard (x_L, x_R).  Returns (lnF, lnG): per shard
    the 2^(l-1) natural logarithms of the forward states at its x_L and the
    backward states at its x_R (entry 0, the empty state, is 0).  FP64 on the
    host: P compositions of 2^(l-1)-vectors."""
    P = len(lnops)
    NS = 1 << (l - 1)
    pc = _popcounts(NS)
    rate = pc * (l - pc)
    lnF, lnG = [None] * P, [None] * P
    cur = np.full(NS, _NEG)
    cur[0] = 0.0
    for q in range(P):
        lnF[q] = cur.copy()
        out = _apply(np.asarray(lnops[q][0]), cur, pc)
        if q + 1 < P:
            cur = out - rate * ((ends[q + 1][0] - ends[q][1]) / eps)
    cur = np.full(NS, _NEG)
    cur[0] = 0.0
    for q in range(P - 1, -1, -1):
        lnG[q] = cur.copy()
        out = _apply(np.asarray(lnops[q][1]), cur, pc)
        if q > 0:
            cur = out - rate * ((ends[q][0] - ends[q - 1][1]) / eps)
    return lnF, lnG


def exchange_distributed(lnop, ends, eps, l, group=None):
    """The exchange with one shard per process: all-gather every rank's
    operator and range ends (ranks in shard order), then the same composition
    on every rank.  Returns this rank's (lnF, lnG)."""
    import torch
    import torch.distributed as dist
    P = dist.get_world_size(group)
    r = dist.get_rank(group)
    mine = torch.from_numpy(np.concatenate([np.asarray(lnop, dtype=np.float64).ravel(),
                                            np.asarray(ends, dtype=np.float64)]))
    parts = [torch.empty_like(mine) for _ in range(P)]
    dist.all_gather(parts, mine, group=group)
    n = mine.numel() - 2
    shape = np.asarray(lnop).shape
    ops = [p.numpy()[:n].reshape(shape) for p in parts]
    ends_all = [tuple(p.numpy()[n:]) for p in parts]
    lnF, lnG = exchange(ops, ends_all, eps, l)
    return lnF[r], lnG[r]


class ShardPlan:
    """One shard's plan (``mmot_shard_create``); N_total: the whole
    instance's sizes."""

    def __init__(self, xs, mus, N_total, eps, precision="fp32"):
        self.l = len(xs)
        xs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in xs]
        mus = [np.ascontiguousarray(np.asarray(m, dtype=np.float64)) for m in mus]
        self.N = [len(x) for x in xs]
        self.eps = float(eps)
        self.ends = range_ends(xs)
        l = self.l
        N_arr = (ctypes.c_int64 * l)(*self.N)
        Nt = (ctypes.c_int64 * l)(*[int(n) for n in N_total])
        X = (ctypes.c_void_p * l)(*[x.ctypes.data for x in xs])
        M = (ctypes.c_void_p * l)(*[m.ctypes.data for m in mus])
        h = ctypes.c_void_p()
        nat.check(nat.lib().mmot_shard_create(l, N_arr, X, M, Nt, self.eps, _PREC[precision], 0, None,
                                              ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().mmot_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def operator(self, k):
        NS = 1 << (self.l - 1)
        out = np.empty((2, self.l, NS), dtype=np.float64)
        nat.check(nat.lib().mmot_shard_operator(self._h, k, out.ctypes.data))
        return out

    def set_inflow(self, k, lnF, lnG):
        f = None if lnF is None else np.ascontiguousarray(lnF, dtype=np.float64)
        g = None if lnG is None else np.ascontiguousarray(lnG, dtype=np.float64)
        nat.check(nat.lib().mmot_shard_set_inflow(self._h, k, None if f is None else f.ctypes.data,
                                                  None if g is None else g.ctypes.data))

    def update(self, k):
        nat.check(nat.lib().mmot_shard_update(self._h, k))

    def residual(self, k):
        r = ctypes.c_double(np.nan)
        nat.check(nat.lib().mmot_shard_residual(self._h, k, ctypes.byref(r)))
        return r.value

    def marginal(self, k, kind="M"):
        res = np.empty(self.N[k], dtype=np.float64)
        nat.check(nat.lib().mmot_marginal(self._h, k, _KIND[kind], res.ctypes.data))
        return res

    def get_potentials(self, k):
        g = np.empty(self.N[k], dtype=np.float64)
        nat.check(nat.lib().mmot_get_potentials(self._h, k, g.ctypes.data))
        return g

    def set_potentials(self, k, g):
        g = np.ascontiguousarray(g, dtype=np.float64)
        nat.check(nat.lib().mmot_set_potentials(self._h, k, g.ctypes.data))


class ShardedPlan:
    """One instance as n_shards shard plans on this GPU with the host
    exchange: products, Gauss-Seidel iterations and the stopping residual
    (marginals 1..l-1, Algorithm 1) give what one plan of the whole instance
    gives."""

    def __init__(self, xs, mus, eps, n_shards, precision="fp32"):
        self.l = len(xs)
        self.eps = float(eps)
        N_total = [len(x) for x in xs]
        self.shards = [ShardPlan(xq, mq, N_total, eps, precision) for xq, mq in split(xs, mus, n_shards)]

    def close(self):
        for s in self.shards:
            s.close()

    def _exchange(self, k):
        ops = [s.operator(k) for s in self.shards]
        lnF, lnG = exchange(ops, [s.ends for s in self.shards], self.eps, self.l)
        for s, f, g in zip(self.shards, lnF, lnG):
            s.set_inflow(k, f, g)

    def marginal(self, k, kind="M"):
        self._exchange(k)
        return np.concatenate([s.marginal(k, kind) for s in self.shards])

    def update(self, k):
        self._exchange(k)
        for s in self.shards:
            s.update(k)

    def sinkhorn_step(self, n_iters=1, residual=False):
        for _ in range(n_iters):
            for k in range(self.l):
                self.update(k)
        if not residual:
            return None
        return self.residual()

    def residual(self):
        tot = 0.0
        for k in range(self.l - 1):
            self._exchange(k)
            tot += sum(s.residual(k) for s in self.shards)
        return tot

    def get_potentials(self, k):
        return np.concatenate([s.get_potentials(k) for s in self.shards])

    def set_potentials(self, k, g):
        off = 0
        for s in self.shards:
            n = s.N[k]
            s.set_potentials(k, np.asarray(g)[off:off + n])
            off += n
