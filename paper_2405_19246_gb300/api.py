"""Python face of the C ABI (``include/mmot.h``): one :class:`Plan` per problem.

Inputs may be numpy arrays (host) or CUDA torch tensors (device); outputs are
numpy arrays unless a CUDA ``out`` tensor is given.  PyTorch is used only for
device memory and streams.  All computation happens in ``libmmot_gb300.so``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat

_PREC = {"fp64": nat.MMOT_FP64, "fp32": nat.MMOT_FP32_SCAN_FP64_POT}
_KIND = {"M": 0, "plan": 1, "lnM": 2}


def _is_cuda_tensor(a):
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _host_f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Plan:
    """An l-marginal L1-cost entropic OT instance resident on the GPU.

    xs, mus: sequences of l supports (sorted) and weights (sum 1); all numpy
    (host) or all CUDA float64 tensors (device).  eps > 0.  precision "fp32"
    (FP32 in-tile scans, FP64 carries and potentials) or "fp64".
    """

    def __init__(self, xs, mus, eps, precision="fp32", stream=None):
        self.l = len(xs)
        if len(mus) != self.l:
            raise ValueError("xs and mus differ in length")
        on_dev = _is_cuda_tensor(xs[0])
        keep = []
        if on_dev:
            import torch
            xs = [x.to(torch.float64).contiguous() for x in xs]
            mus = [m.to(torch.float64).contiguous() for m in mus]
            xp = [x.data_ptr() for x in xs]
            mp = [m.data_ptr() for m in mus]
            Ns = [x.numel() for x in xs]
            keep = xs + mus
        else:
            xs = [_host_f64(x) for x in xs]
            mus = [_host_f64(m) for m in mus]
            xp = [x.ctypes.data for x in xs]
            mp = [m.ctypes.data for m in mus]
            Ns = [len(x) for x in xs]
            keep = xs + mus
        self.N = Ns
        self.eps = float(eps)
        self.precision = precision
        N_arr = (ctypes.c_int64 * self.l)(*Ns)
        X = (ctypes.c_void_p * self.l)(*xp)
        M = (ctypes.c_void_p * self.l)(*mp)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        nat.check(nat.lib().mmot_plan_create(self.l, N_arr, X, M, self.eps, _PREC[precision],
                                             1 if on_dev else 0, st, ctypes.byref(h)))
        del keep
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            nat.lib().mmot_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------
    def marginal(self, k, kind="M", out=None):
        """M_k (kind "M"), phi_k M_k ("plan") or ln M_k ("lnM")."""
        if out is None:
            res = np.empty(self.N[k], dtype=np.float64)
            nat.check(nat.lib().mmot_marginal(self._h, k, _KIND[kind], res.ctypes.data))
            return res
        nat.check(nat.lib().mmot_marginal(self._h, k, _KIND[kind], out.data_ptr()))
        return out

    def sinkhorn_step(self, n_iters=1, residual=False):
        r = ctypes.c_double(np.nan)
        nat.check(nat.lib().mmot_sinkhorn_step(self._h, int(n_iters),
                                               ctypes.byref(r) if residual else None))
        return r.value if residual else None

    def solve(self, tol, itr_max, allow_not_converged=True):
        res = nat.MmotResult()
        st = nat.lib().mmot_solve(self._h, float(tol), int(itr_max), ctypes.byref(res))
        if not (st == nat.MMOT_OK or (allow_not_converged and st == 6)):
            nat.check(st)
        return dict(iters=res.iters, residual=res.residual, W=res.W, primal=res.primal,
                    dual=res.dual, mass=res.mass, converged=(st == nat.MMOT_OK))

    def objective(self):
        res = nat.MmotResult()
        nat.check(nat.lib().mmot_objective(self._h, ctypes.byref(res)))
        return dict(residual=res.residual, W=res.W, primal=res.primal, dual=res.dual, mass=res.mass)

    def get_potentials(self, k, out=None):
        if out is None:
            g = np.empty(self.N[k], dtype=np.float64)
            nat.check(nat.lib().mmot_get_potentials(self._h, k, g.ctypes.data))
            return g
        nat.check(nat.lib().mmot_get_potentials(self._h, k, out.data_ptr()))
        return out

    def set_potentials(self, k, g):
        if _is_cuda_tensor(g):
            nat.check(nat.lib().mmot_set_potentials(self._h, k, g.contiguous().data_ptr()))
        else:
            g = _host_f64(g)
            nat.check(nat.lib().mmot_set_potentials(self._h, k, g.ctypes.data))

    def reset_potentials(self):
        nat.check(nat.lib().mmot_reset_potentials(self._h))

    def profile(self, on=True):
        nat.check(nat.lib().mmot_set_option(self._h, nat.MMOT_OPT_PROFILE, 1 if on else 0))

    def profile_stats(self, reset=True):
        """{kernel name: (launches, total ms)} from the CUDA-event profile."""
        out = {}
        names = ((0, "k_bwd"), (1, "k_fwd"), (2, "k_tops"), (3, "k_carry"),
                 (4, "k_tile" if self.l <= 5 else "k_wprod"), (5, "k_wpass"), (6, "k_lscan"), (7, "k_wbwd"))
        for k, name in names:
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            nat.check(nat.lib().mmot_get_profile(self._h, k, ctypes.byref(n), ctypes.byref(ms),
                                                 1 if (reset and k == 7) else 0))
            out[name] = (n.value, ms.value)
        return out

    def set_option(self, option, value):
        nat.check(nat.lib().mmot_set_option(self._h, int(option), int(value)))

    def info(self):
        inf = nat.MmotPlanInfo()
        nat.check(nat.lib().mmot_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}


class Batch:
    """Many independent instances solved together (host inputs).

    instances: sequence of (xs, mus, eps) with xs, mus sequences of l numpy
    arrays each (l may differ between instances).  Instances with the same l
    share one launch sequence; each instance is frozen once its residual is
    at most tol at a check.
    """

    def __init__(self, instances, precision="fp32", tile_points=0, stream=None):
        ls, Ns, xp, mp, eps, keep = [], [], [], [], [], []
        for xs, mus, e in instances:
            if len(xs) != len(mus):
                raise ValueError("xs and mus differ in length")
            ls.append(len(xs))
            for x, m in zip(xs, mus):
                x = _host_f64(x)
                m = _host_f64(m)
                keep += [x, m]
                Ns.append(len(x))
                xp.append(x.ctypes.data)
                mp.append(m.ctypes.data)
            eps.append(float(e))
        self.n = len(ls)
        self.l = ls
        self.N = []
        o = 0
        for li in ls:
            self.N.append(Ns[o:o + li])
            o += li
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        nat.check(nat.lib().mmot_batch_create(
            self.n, (ctypes.c_int * self.n)(*ls), (ctypes.c_int64 * len(Ns))(*Ns),
            (ctypes.c_void_p * len(xp))(*xp), (ctypes.c_void_p * len(mp))(*mp),
            (ctypes.c_double * self.n)(*eps), _PREC[precision], int(tile_points), st, ctypes.byref(h)))
        del keep
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().mmot_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self):
        nat.check(nat.lib().mmot_batch_reset(self._h))

    def step(self, n_iters, tol):
        """n_iters iterations on the running instances, then a check; returns
        the number of instances still running."""
        a = ctypes.c_int()
        nat.check(nat.lib().mmot_batch_step(self._h, int(n_iters), float(tol), ctypes.byref(a)))
        return a.value

    def solve(self, tol, itr_max, check_every=10, results=True):
        """Solve all instances; list of per-instance result dicts (or None)."""
        arr = (nat.MmotResult * self.n)() if results else None
        st = nat.lib().mmot_batch_solve(self._h, float(tol), int(itr_max), int(check_every), arr)
        if st not in (nat.MMOT_OK, 6):
            nat.check(st)
        if not results:
            return None
        return [dict(iters=r.iters, residual=r.residual, W=r.W, primal=r.primal, dual=r.dual,
                     mass=r.mass) for r in arr]

    def freeze(self, i):
        """Stop updating instance i (its iteration budget is spent)."""
        nat.check(nat.lib().mmot_batch_freeze(self._h, int(i)))

    def status(self, i):
        it, res, cv = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        nat.check(nat.lib().mmot_batch_status(self._h, int(i), ctypes.byref(it), ctypes.byref(res),
                                              ctypes.byref(cv)))
        return dict(iters=it.value, residual=res.value, converged=bool(cv.value))

    def get_potentials(self, i, k):
        g = np.empty(self.N[i][k], dtype=np.float64)
        nat.check(nat.lib().mmot_batch_get_potentials(self._h, int(i), int(k), g.ctypes.data))
        return g

    def set_potentials(self, i, k, g):
        """Replace g_k of instance i (a warm start; see mmot_batch_set_potentials)."""
        g = np.ascontiguousarray(g, dtype=np.float64)
        if g.shape != (self.N[i][k],):
            raise ValueError("instance %d, marginal %d takes %d potentials" % (i, k, self.N[i][k]))
        nat.check(nat.lib().mmot_batch_set_potentials(self._h, int(i), int(k), g.ctypes.data))

    def info(self):
        inf = nat.MmotBatchInfo()
        nat.check(nat.lib().mmot_batch_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}


def ftvp2d(phi, psi, lambda1, lambda2):
    """Two-dimensional product of three marginals on one uniform grid
    (``mmot_ftvp2d``; Sec. 4.1, Algorithm 6): out = K x phi x psi for the
    separable L1 kernel with lambda_d = exp(-h_d / eps).  phi, psi: (N, M)
    arrays (numpy) indexed [i1, i2]; returns an (N, M) numpy array."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    if phi.shape != psi.shape or phi.ndim != 2:
        raise ValueError("phi and psi must be (N, M) arrays of the same shape")
    N, M = phi.shape
    # column-major: element (i1, i2) at i1 + N i2
    a = np.ascontiguousarray(phi.T)
    b = np.ascontiguousarray(psi.T)
    out = np.empty((M, N), dtype=np.float64)
    nat.check(nat.lib().mmot_ftvp2d(N, M, a.ctypes.data, b.ctypes.data, float(lambda1), float(lambda2),
                                    out.ctypes.data, None))
    return out.T.copy()
