"""Plain FP64 CPU oracle for multi-marginal Sinkhorn with pairwise L1 cost.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it
and shares no code with it.

Two independent implementations live here:

* ``brute`` (this package, numpy): the dense tensor definition, O(N^l).
  M_j(i) = sum over the other marginals' points of prod phi * exp(-c/eps)
  with c = sum_{p<q} |y_p - y_q| (Sec. 4.2, Eq. Jk k margin) and
  W = sum c * t (Eq. k-mmot distance).
* ``mmot_oracle.c`` (compiled to ``liboracle_mmot.so`` by ``build()``):
  the paper's order-class chains (Sec. 4.2), the subset-state form of the
  same chains, the literal l = 3 uniform-grid Algorithms 2, 3 and 4, and a
  log-domain Gauss-Seidel Sinkhorn driver (Sec. 4.2 update formulas).

All potentials are g_k = eps ln phi_k.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmot_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_mmot.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i64, i = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        pd = P(d)
        ppd = P(pd)
        L.mo_merge.argtypes = [i, P(i64), ppd, P(i), P(i64)]
        L.mo_marginal_classes.argtypes = [i, P(i64), ppd, ppd, d, i, pd]
        L.mo_marginal_subset.argtypes = [i, P(i64), ppd, ppd, d, i, pd]
        L.mo_marginal_subset_sel.argtypes = [i, P(i64), ppd, ppd, d, i, i64, P(i64), pd]
        L.mo_allpass.argtypes = [i, P(i64), ppd, ppd, d, ppd, pd, pd]
        L.mo_ftvp1.argtypes = [i64, pd, pd, d, pd]
        L.mo_ftvp1.restype = None
        L.mo_ftvp2.argtypes = [i64, pd, pd, d, d, pd]
        L.mo_ftvp2.restype = None
        L.mo_fs3.argtypes = [i64, pd, pd, pd, d, d, d, i, pd, pd, pd, pd, P(i), pd]
        L.mo_sinkhorn.argtypes = [i, P(i64), ppd, ppd, d, d, i, ppd, P(i), pd, pd, pd, pd, pd]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr_array(arrs):
    arr_t = ctypes.POINTER(ctypes.c_double) * len(arrs)
    return arr_t(*[_dptr(a) for a in arrs])


def _sizes(xs):
    return (ctypes.c_int64 * len(xs))(*[len(x) for x in xs])


def merge(xs):
    """Merged order (marginal id, local index) by the key (x, k, i)."""
    xs = [_f64(x) for x in xs]
    T = sum(len(x) for x in xs)
    mid = np.zeros(T, dtype=np.int32)
    loc = np.zeros(T, dtype=np.int64)
    rc = lib().mo_merge(len(xs), _sizes(xs), _ptr_array(xs),
                        mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        loc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc:
        raise ValueError("unsorted support")
    return mid, loc


def marginal_classes(xs, gs, eps, j):
    """ln M_j by the l! order-class chains (Sec. 4.2)."""
    xs = [_f64(x) for x in xs]
    gs = [_f64(g) for g in gs]
    out = np.empty(len(xs[j]))
    rc = lib().mo_marginal_classes(len(xs), _sizes(xs), _ptr_array(xs), _ptr_array(gs),
                                   float(eps), int(j), _dptr(out))
    if rc:
        raise RuntimeError("oracle error %d" % rc)
    return out


def marginal_subset(xs, gs, eps, j, want=None):
    """ln M_j by the subset-state chains; optionally only at j-points ``want``."""
    xs = [_f64(x) for x in xs]
    gs = [_f64(g) for g in gs]
    if want is None:
        out = np.empty(len(xs[j]))
        rc = lib().mo_marginal_subset(len(xs), _sizes(xs), _ptr_array(xs), _ptr_array(gs),
                                      float(eps), int(j), _dptr(out))
    else:
        w = np.ascontiguousarray(np.asarray(want, dtype=np.int64))
        if np.any(np.diff(w) <= 0):
            raise ValueError("want must be strictly increasing")
        out = np.empty(len(w))
        rc = lib().mo_marginal_subset_sel(len(xs), _sizes(xs), _ptr_array(xs), _ptr_array(gs),
                                          float(eps), int(j), len(w),
                                          w.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          _dptr(out))
    if rc:
        raise RuntimeError("oracle error %d" % rc)
    return out


def allpass(xs, gs, eps):
    """(list of ln M_k, ln Z, W) from one all-subset sweep pair."""
    xs = [_f64(x) for x in xs]
    gs = [_f64(g) for g in gs]
    outs = [np.empty(len(x)) for x in xs]
    lnZ = ctypes.c_double()
    W = ctypes.c_double()
    rc = lib().mo_allpass(len(xs), _sizes(xs), _ptr_array(xs), _ptr_array(gs), float(eps),
                          _ptr_array(outs), ctypes.byref(lnZ), ctypes.byref(W))
    if rc:
        raise RuntimeError("oracle error %d" % rc)
    return outs, lnZ.value, W.value


def ftvp1(phi, psi, lam):
    """Algorithm 2 (FTVP-1)."""
    phi, psi = _f64(phi), _f64(psi)
    out = np.empty(len(phi))
    lib().mo_ftvp1(len(phi), _dptr(phi), _dptr(psi), float(lam), _dptr(out))
    return out


def ftvp2(phi, psi, lam, h):
    """Algorithm 3 (FTVP-2) with the factor N in R_{N,5}, R_{N,6}."""
    phi, psi = _f64(phi), _f64(psi)
    out = np.empty(len(phi))
    lib().mo_ftvp2(len(phi), _dptr(phi), _dptr(psi), float(lam), float(h), _dptr(out))
    return out


def fs3(u, v, w, h, eps, tol, itr_max):
    """Algorithm 4; returns dict with phi, psi, varphi, W, iters, res."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    N = len(u)
    phi, psi, vphi = np.empty(N), np.empty(N), np.empty(N)
    W = ctypes.c_double()
    it = ctypes.c_int()
    res = ctypes.c_double()
    lib().mo_fs3(N, _dptr(u), _dptr(v), _dptr(w), float(h), float(eps), float(tol), int(itr_max),
                 _dptr(phi), _dptr(psi), _dptr(vphi), ctypes.byref(W), ctypes.byref(it),
                 ctypes.byref(res))
    return dict(phi=phi, psi=psi, varphi=vphi, W=W.value, iters=it.value, res=res.value)


def sinkhorn(xs, mus, eps, tol, itr_max, g0=None):
    """Log-domain Gauss-Seidel Sinkhorn for general l.

    Starts from phi = 1/N_k (g = -eps ln N_k) unless ``g0`` is given.
    Returns dict with g (list), iters, res, W, primal, dual, mass.
    """
    xs = [_f64(x) for x in xs]
    mus = [_f64(m) for m in mus]
    if g0 is None:
        gs = [np.full(len(x), -eps * np.log(len(x))) for x in xs]
    else:
        gs = [np.array(g, dtype=np.float64, copy=True) for g in g0]
    it = ctypes.c_int()
    res, W, P, D, Z = (ctypes.c_double() for _ in range(5))
    rc = lib().mo_sinkhorn(len(xs), _sizes(xs), _ptr_array(xs), _ptr_array(mus), float(eps),
                           float(tol), int(itr_max), _ptr_array(gs), ctypes.byref(it),
                           ctypes.byref(res), ctypes.byref(W), ctypes.byref(P), ctypes.byref(D),
                           ctypes.byref(Z))
    if rc:
        raise RuntimeError("oracle error %d" % rc)
    return dict(g=gs, iters=it.value, res=res.value, W=W.value, primal=P.value,
                dual=D.value, mass=Z.value)


def potential_update(mu, lnM, eps):
    """g_j = eps (ln mu_j - ln M_j); a zero weight gives -inf (Sec. 4.2 updates)."""
    mu = np.asarray(mu, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(mu > 0, eps * (np.log(np.where(mu > 0, mu, 1.0)) - lnM), -np.inf)
