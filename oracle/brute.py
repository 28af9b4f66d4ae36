"""Dense-tensor definition of the l-marginal products (tiny inputs only).

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is the plain O(N^l) definition that the fast method must reproduce
exactly (Sec. 4.2, Eq. Jk k margin and Eq. k-mmot distance; Algorithm 1 is the
generalized Sinkhorn that uses these dense products):

    c(y_1..y_l) = sum_{p<q} |y_p - y_q|
    ln t        = sum_k g_k(y_k)/eps - c/eps
    ln M_j(i)   = logsumexp over all tuples with i_j = i of
                  sum_{m != j} g_m(y_m)/eps - c/eps
    W           = sum over tuples of c * t

It shares nothing with the C oracle.  The tensor has prod_k N_k entries, so
keep that product below a few million.
"""
from __future__ import annotations

import numpy as np


def _logsumexp(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(a - m), axis=axis))


def cost_tensor(xs):
    """Dense pairwise-L1 cost tensor, shape (N_1, ..., N_l)."""
    l = len(xs)
    grids = np.meshgrid(*[np.asarray(x, dtype=np.float64) for x in xs], indexing="ij")
    C = np.zeros(grids[0].shape)
    for p in range(l):
        for q in range(p + 1, l):
            C += np.abs(grids[p] - grids[q])
    return C


def _potential_sum(gs, eps, skip=None):
    l = len(gs)
    shape = tuple(len(g) for g in gs)
    S = np.zeros(shape)
    for k in range(l):
        if k == skip:
            continue
        sh = [1] * l
        sh[k] = shape[k]
        S = S + np.asarray(gs[k], dtype=np.float64).reshape(sh) / eps
    return S


def ln_marginal_product(xs, gs, eps, j):
    """ln M_j(i) for every point i of marginal j by the dense definition."""
    C = cost_tensor(xs)
    A = _potential_sum(gs, eps, skip=j) - C / eps
    axes = tuple(k for k in range(len(xs)) if k != j)
    B = np.moveaxis(A, j, 0).reshape(len(xs[j]), -1)
    del axes
    return _logsumexp(B, axis=1)


def plan(xs, gs, eps):
    """Dense plan t = prod_k phi_k K (Eq. k-marginal T value)."""
    C = cost_tensor(xs)
    return np.exp(_potential_sum(gs, eps) - C / eps)


def transport_cost(xs, gs, eps):
    """W = <C, T> (Eq. k-mmot distance)."""
    C = cost_tensor(xs)
    return float(np.sum(C * np.exp(_potential_sum(gs, eps) - C / eps)))


def sinkhorn_dense(xs, mus, eps, n_iter, g0=None):
    """Algorithm 1 / Sec. 4.2 Gauss-Seidel updates with dense products.

    Returns the potentials after ``n_iter`` full iterations from phi = 1/N_k.
    """
    gs = ([np.full(len(x), -eps * np.log(len(x))) for x in xs] if g0 is None
          else [np.array(g, dtype=np.float64) for g in g0])
    for _ in range(n_iter):
        for j in range(len(xs)):
            lnM = ln_marginal_product(xs, gs, eps, j)
            mu = np.asarray(mus[j], dtype=np.float64)
            with np.errstate(divide="ignore"):
                gs[j] = np.where(mu > 0, eps * (np.log(np.where(mu > 0, mu, 1.0)) - lnM), -np.inf)
    return gs
