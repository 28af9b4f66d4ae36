"""Seeded synthetic inputs for l-marginal optimal transport with L1 cost.

This module only draws inputs (supports x_k and weights mu_k); it holds none
of the method's arithmetic.  Both the CUDA path and the CPU oracle are fed
from here.

Every marginal is drawn from its own stream,
``numpy.random.default_rng(SeedSequence([config_id, instance, marginal]))``,
and only ``Generator.random`` (uniform doubles) is used; normals and
exponentials are derived from the uniforms here (Box-Muller, -ln U) so that
the draws do not depend on numpy's sampler internals.

Workloads (sizes and laws follow the paper's experiments, Sec. 5, and the
benchmark configurations of this library):

* ``uniform_grid_mixture``  uniform grid on [0, 1] (x_i = i/(N-1)), weights a
  two-component Gaussian mixture (means U[0.2, 0.8], sd U[0.05, 0.15], equal
  component weights) evaluated on the grid and normalised.
* ``sorted_uniform_lognormal``  x = sort(U[0,1]^N), weights LogNormal(0, 1)
  normalised.
* ``sorted_uniform_dirichlet``  x = sort(U[0,1]^N), weights Dirichlet(1)
  (normalised Exp(1)).
* ``paper_random_1d``  the 1-D random distributions of Sec. 5.1: uniform grid
  on [0, 1], weights U[0, 1] normalised.
* ``paper_ricker``  the Ricker wavelets of Sec. 5.2 (see the function).
* ``batched_instances``  independent instances with l uniform in {3..8}, N
  log-uniform in [64, 65536], eps log-uniform in [1e-3, 1e-1], sorted U[0,1]
  supports and LogNormal(0, 1) weights.
"""
from __future__ import annotations

import math

import numpy as np

# configuration ids used as the first seed word
CFG_GRID_MIXTURE = 1
CFG_LOGNORMAL = 2
CFG_DIRICHLET = 3
CFG_BATCHED = 4
CFG_SERVING = 5
CFG_PAPER_RANDOM = 11
CFG_PAPER_RICKER = 12
CFG_TEST = 99


def _rng(cfg, instance, marginal):
    return np.random.default_rng(np.random.SeedSequence([int(cfg), int(instance), int(marginal)]))


def _normals(rng, n):
    """Standard normals by Box-Muller from uniform doubles."""
    m = (n + 1) // 2
    u1 = 1.0 - rng.random(m)        # (0, 1]
    u2 = rng.random(m)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def _exponentials(rng, n):
    return -np.log(1.0 - rng.random(n))


def uniform_grid_mixture(l=3, N=1000, seed_cfg=CFG_GRID_MIXTURE, instance=0):
    xs, mus = [], []
    x = np.linspace(0.0, 1.0, N) if N > 1 else np.zeros(1)
    for k in range(l):
        rng = _rng(seed_cfg, instance, k)
        means = 0.2 + 0.6 * rng.random(2)
        sds = 0.05 + 0.10 * rng.random(2)
        dens = np.zeros(N)
        for c in range(2):
            dens += 0.5 * np.exp(-0.5 * ((x - means[c]) / sds[c]) ** 2) / (sds[c] * math.sqrt(2 * math.pi))
        xs.append(x.copy())
        mus.append(dens / dens.sum())
    return xs, mus


def sorted_uniform_lognormal(l=4, N=1 << 20, seed_cfg=CFG_LOGNORMAL, instance=0, Ns=None):
    xs, mus = [], []
    for k in range(l):
        n = N if Ns is None else int(Ns[k])
        rng = _rng(seed_cfg, instance, k)
        x = np.sort(rng.random(n))
        w = np.exp(_normals(rng, n))
        xs.append(x)
        mus.append(w / w.sum())
    return xs, mus


def sorted_uniform_dirichlet(l=8, N=1 << 24, seed_cfg=CFG_DIRICHLET, instance=0):
    xs, mus = [], []
    for k in range(l):
        rng = _rng(seed_cfg, instance, k)
        x = np.sort(rng.random(N))
        w = _exponentials(rng, N)
        xs.append(x)
        mus.append(w / w.sum())
    return xs, mus


def paper_random_1d(N, instance=0, l=3):
    """Sec. 5.1: grid points uniformly spaced on [0,1], weights U[0,1] normalised."""
    x = np.linspace(0.0, 1.0, N)
    xs, mus = [], []
    for k in range(l):
        rng = _rng(CFG_PAPER_RANDOM, instance, k)
        u = rng.random(N)
        xs.append(x.copy())
        mus.append(u / u.sum())
    return xs, mus


def paper_ricker(N, delta=1e-3, A=1.0, F0=1.0, taus=(0.0, 0.75, 1.5)):
    """Sec. 5.2: Ricker wavelets f_k(t) = R(t - tau_k) with
    R(t) = A (1 - 2 pi^2 F0^2 t^2) exp(-pi^2 F0^2 t^2) on a uniform grid on
    [-2, 2], turned into weights by (f^2/||f^2||_1 + delta)/(1 + L delta) with
    L = N, which makes every weight vector sum to one."""
    x = np.linspace(-2.0, 2.0, N)
    xs, mus = [], []
    for tau in taus:
        t = x - tau
        f = A * (1.0 - 2.0 * math.pi ** 2 * F0 ** 2 * t ** 2) * np.exp(-(math.pi ** 2) * F0 ** 2 * t ** 2)
        f2 = f * f
        w = (f2 / f2.sum() + delta) / (1.0 + N * delta)
        xs.append(x.copy())
        mus.append(w)
    return xs, mus


def batched_instance_params(count, seed_cfg=CFG_BATCHED, l_range=(3, 8), N_range=(64, 65536),
                            eps_range=(1e-3, 1e-1)):
    """(l, N, eps) per instance: l uniform in l_range, N and eps log-uniform."""
    rng = _rng(seed_cfg, 1 << 30, 0)
    u = rng.random((count, 3))
    lo, hi = l_range
    ls = lo + np.minimum((u[:, 0] * (hi - lo + 1)).astype(np.int64), hi - lo)
    Ns = np.rint(np.exp(math.log(N_range[0]) + u[:, 1] * (math.log(N_range[1]) - math.log(N_range[0]))))
    eps = np.exp(math.log(eps_range[0]) + u[:, 2] * (math.log(eps_range[1]) - math.log(eps_range[0])))
    return [(int(a), int(b), float(c)) for a, b, c in zip(ls, Ns.astype(np.int64), eps)]


def batched_instance(index, l, N, seed_cfg=CFG_BATCHED):
    """Inputs of one batched instance: sorted U[0,1] supports, LogNormal(0,1) weights."""
    return sorted_uniform_lognormal(l=l, N=N, seed_cfg=seed_cfg, instance=index)


def random_small(l, Ns, seed=0, ties=False, zeros=False, grid=None):
    """Small test instances: sorted U[0,1] supports (or points on a shared grid
    of ``grid`` values when ``ties``), LogNormal weights, optional zero weights."""
    xs, mus = [], []
    for k in range(l):
        rng = _rng(CFG_TEST, seed, k)
        n = int(Ns[k])
        if ties:
            G = grid if grid is not None else max(2, n // 2)
            x = np.sort(np.floor(rng.random(n) * G) / G)
        else:
            x = np.sort(rng.random(n))
        w = np.exp(_normals(rng, n))
        if zeros and n > 2:
            w[rng.random(n) < 0.25] = 0.0
            if w.sum() == 0:
                w[0] = 1.0
        xs.append(x)
        mus.append(w / w.sum())
    return xs, mus
