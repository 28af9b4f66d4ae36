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


# ---- transfer operator of a range of the merged order (shards) ---------------
# For sorted points the pairwise L1 cost of one point per marginal is a sum
# over the gaps between consecutive merged positions: a gap of length d with
# s of the chosen points on its left costs d * s (l - s) (each of the s
# points pairs with each of the l - s points on the right).  A partial
# placement of the marginals in S left of x therefore carries
# exp(-sum_{gaps left of x} d * w(#S-points left of the gap)/eps), w(s) =
# s(l - s): the subset states of Sec. 4.2.  Over a range (x_L, x_R] of the
# merged order a state S of level s picks up the points of the marginals in U
# one at a time, each point adding its phi and raising the rate of the gaps
# after it.  Brute force over the placements of U inside the range.


def merged_order(xs):
    """Merged order of all points: sorted by x, then marginal, then index.
    Returns (x, marginal, index) arrays in that order."""
    X = np.concatenate([np.asarray(x, dtype=np.float64) for x in xs])
    K = np.concatenate([np.full(len(x), k) for k, x in enumerate(xs)])
    I = np.concatenate([np.arange(len(x)) for x in xs])
    o = np.lexsort((I, K, X))
    return X[o], K[o], I[o]


def state_bits(l, j):
    """Marginal of each state bit for target j (bit b: marginal b if b < j,
    else b + 1)."""
    return [m for m in range(l) if m != j]


def range_operator(xs, gs, eps, j, lo, hi, x_start, x_end, backward=False):
    """ln op[s][U] of the merged positions lo..hi-1 for target j.

    Forward: a state of level s at x_start (left of position lo) reaching
    S + U at x_end (right of position hi - 1); backward: the mirror image,
    from x_end down to x_start.  op[s][0] = -w(s) (x_end - x_start)/eps.
    Entries with s + |U| > l - 1 are -inf.  Shape [l, 2^(l-1)]."""
    l = len(xs)
    X, K, I = merged_order(xs)
    bits = state_bits(l, j)
    NB = l - 1
    NS = 1 << NB
    w = [s * (l - s) for s in range(l + 1)]
    out = np.full((l, NS), -np.inf)
    span = x_end - x_start
    for s in range(l):
        out[s, 0] = -w[s] * span / eps
    pts = {m: [t for t in range(lo, hi) if K[t] == m] for m in range(l)}
    import itertools
    for s in range(NB):
        for U in range(1, NS):
            mU = [bits[b] for b in range(NB) if (U >> b) & 1]
            if s + len(mU) > NB:
                continue
            terms = []
            for choice in itertools.product(*[pts[m] for m in mU]):
                ps = sorted(choice)
                lnphi = sum(gs[K[t]][I[t]] / eps for t in ps)
                if backward:
                    ps = ps[::-1]
                    edges = [x_end] + [X[t] for t in ps] + [x_start]
                    cost = sum(w[s + i] * (edges[i] - edges[i + 1]) for i in range(len(ps) + 1))
                else:
                    edges = [x_start] + [X[t] for t in ps] + [x_end]
                    cost = sum(w[s + i] * (edges[i + 1] - edges[i]) for i in range(len(ps) + 1))
                terms.append(lnphi - cost / eps)
            if terms:
                t = np.array(terms)
                m = np.max(t)
                out[s, U] = m + np.log(np.sum(np.exp(t - m))) if np.isfinite(m) else -np.inf
    return out


def apply_operator(op, lnin):
    """ln of the states leaving a range, out[T] = logsumexp_{S inside T}
    lnin[S] + op[|S|][T \\ S] (lnin[0] = 0: the empty state)."""
    NS = len(lnin)
    out = np.full(NS, -np.inf)
    for T in range(NS):
        terms = []
        for S in range(NS):
            if (S & ~T) == 0 and lnin[S] > -np.inf and op[bin(S).count("1"), T ^ S] > -np.inf:
                terms.append(lnin[S] + op[bin(S).count("1"), T ^ S])
        if terms:
            t = np.array(terms)
            m = np.max(t)
            out[T] = m + np.log(np.sum(np.exp(t - m)))
    return out


def ln_marginal_in_range(xs, gs, eps, j, lo, hi, lnF_in, lnG_in, x_L, x_R):
    """ln M_j at the points of marginal j among merged positions lo..hi-1,
    from the states entering the range (forward at x_L, backward at x_R) and
    the range's own points: M_j(i) = sum_S F_S(x_i^-) G_{R \\ S}(x_i^+) (the
    combine of Sec. 4.2)."""
    l = len(xs)
    X, K, _ = merged_order(xs)
    NS = 1 << (l - 1)
    full = NS - 1
    res = []
    for t in range(lo, hi):
        if K[t] != j:
            continue
        F = apply_operator(range_operator(xs, gs, eps, j, lo, t, x_L, X[t]), lnF_in)
        G = apply_operator(range_operator(xs, gs, eps, j, t + 1, hi, X[t], x_R, backward=True), lnG_in)
        terms = np.array([F[S] + G[full ^ S] for S in range(NS)])
        m = np.max(terms)
        res.append(m + np.log(np.sum(np.exp(terms - m))) if np.isfinite(m) else -np.inf)
    return np.array(res)


# ---- the two-dimensional product (Sec. 4.1) -----------------------------------


def kernel_1d(n, lam):
    """K(i, j, k) = lam^{|i-j| + |i-k| + |j-k|} on a uniform grid of n points."""
    i = np.arange(n)
    e = (np.abs(i[:, None, None] - i[None, :, None]) + np.abs(i[:, None, None] - i[None, None, :])
         + np.abs(i[None, :, None] - i[None, None, :]))
    return np.power(float(lam), e)


def ftvp2d_dense(phi, psi, lam1, lam2):
    """The two-dimensional product by its definition (Sec. 4.1, Eq. J_{k1k2}):
    J(k1, k2) = sum over i1, i2, j1, j2 of K1(i1, j1, k1) K2(i2, j2, k2)
    phi(i1, i2) psi(j1, j2), with the L1 kernel of each axis.  O(N^3 M^3)."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    N, M = phi.shape
    return np.einsum("abk,cdl,ac,bd->kl", kernel_1d(N, lam1), kernel_1d(M, lam2), phi, psi)
