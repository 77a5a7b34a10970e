"""User-facing wrapper over the C ABI.  Device memory comes from PyTorch; every
step of the computation runs in libewh.so (there is no CPU path: without a
CUDA device, creating a context raises)."""
from __future__ import annotations

import numpy as np

from . import _lib as L


def make_desc(dim, n, h, order, bc, precision=L.EWH_FP64, cfl=0.5, periods=1, corrected=1, nt=0, implicit=0):
    d = L.ewh_grid_desc()
    d.dim = int(dim)
    for a in range(3):
        d.n[a] = int(n[a]) if a < dim else 1
    d.h = float(h)
    d.order = int(order)
    bc = list(bc) + [0] * (6 - len(bc))
    for k in range(6):
        d.bc[k] = int(bc[k])
    d.precision = int(precision)
    d.cfl = float(cfl)
    d.periods = int(periods)
    d.corrected = int(corrected)
    d.nt = int(nt)
    d.implicit = int(implicit)
    return d


PRECISIONS = {"fp64": L.EWH_FP64, "fp32": L.EWH_FP32_STENCIL}


class WaveHoltz:
    """One El-WaveHoltz problem (medium, frequency, forcing) on the current GPU."""

    def __init__(self, prob, precision="fp64", nt=0, stream=None, forcing=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("WaveHoltz needs a CUDA device (libewh.so has no CPU path)")
        self.torch = torch
        self.prob = prob
        self.precision = precision
        desc = make_desc(prob.dim, prob.n, prob.h, prob.order, prob.bc, PRECISIONS[precision],
                         prob.cfl, prob.periods, prob.corrected, nt, getattr(prob, "implicit", 0))
        rho = np.ascontiguousarray(prob.rho, dtype=np.float64)
        lam = np.ascontiguousarray(prob.lam, dtype=np.float64)
        mu = np.ascontiguousarray(prob.mu, dtype=np.float64)
        f = np.ascontiguousarray(prob.forcing, dtype=np.float64) if forcing else None
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        mapping = getattr(prob, "mapping", None)
        if mapping is not None:  # curvilinear grid: node coordinates (x, y)
            X = np.ascontiguousarray(mapping[0], dtype=np.float64)
            Y = np.ascontiguousarray(mapping[1], dtype=np.float64)
            self.ctx = L.ewh_create_mapped(desc, X, Y, rho, lam, mu, prob.omega, f, prob.nrhs, s)
        else:
            self.ctx = L.ewh_create(desc, rho, lam, mu, prob.omega, f, prob.nrhs, s)
        self.info = L.ewh_get_info(self.ctx)
        self.nrhs = prob.nrhs
        self.n = int(self.info.n_unknowns) * prob.nrhs

    # -- helpers
    def _vec(self, x=None):
        t = self.torch
        if x is None:
            return t.empty(self.n, dtype=t.float64, device="cuda")
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
        return x.to(device="cuda", dtype=t.float64).contiguous().reshape(-1)

    def apply_S(self, v, fp64=False):
        v = self._vec(v)
        out = self._vec()
        (L.ewh_apply_S_fp64 if fp64 else L.ewh_apply_S)(self.ctx, v, out)
        return out

    def apply_Pi0(self):
        out = self._vec()
        L.ewh_apply_Pi0(self.ctx, out)
        return out

    def apply_minvK(self, u):
        u = self._vec(u)
        out = self._vec()
        L.ewh_apply_minvK(self.ctx, u, out)
        return out

    def mdot(self, x, y):
        return L.ewh_mdot(self.ctx, self._vec(x), self._vec(y), self.nrhs)

    def solve(self, tol=1e-8, maxit=100000, x0=None, raise_on_error=True):
        out = self._vec()
        x0v = self._vec(x0) if x0 is not None else None
        info = L.ewh_solve(self.ctx, tol, maxit, x0v, out, raise_on_error=raise_on_error)
        return out, info

    def solve_cr(self, tol=1e-8, maxit=100000, x0=None, raise_on_error=True):
        """Conjugate residual instead of CG (non-increasing residual)."""
        out = self._vec()
        x0v = self._vec(x0) if x0 is not None else None
        info = L.ewh_solve_cr(self.ctx, tol, maxit, x0v, out, raise_on_error=raise_on_error)
        return out, info

    def solve_minres(self, tol=1e-8, maxit=100000, x0=None, raise_on_error=True):
        """MINRES instead of CG: for systems that may be indefinite (few time
        steps per period near a resonance); the residual never increases."""
        out = self._vec()
        x0v = self._vec(x0) if x0 is not None else None
        info = L.ewh_solve_minres(self.ctx, tol, maxit, x0v, out, raise_on_error=raise_on_error)
        return out, info

    def residual_history(self):
        return L.ewh_residual_history(self.ctx)

    def kernel_launches(self):
        return L.ewh_kernel_launches(self.ctx)

    def stats(self):
        return L.ewh_get_stats(self.ctx)

    def reset_stats(self):
        L.ewh_reset_stats(self.ctx)

    def set_grid_wait(self, ns):
        """Bound of each grid-barrier wait of the on-chip wave solve, in ns
        (0: every wait gives up at once)."""
        L.ewh_set_grid_wait(self.ctx, ns)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            self.torch.cuda.synchronize()
            L.ewh_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WaveHoltzBatch:
    """Independent problems (shots, frequencies, sizes) solved together: one
    CUDA graph per CG iteration with a branch per unconverged member."""

    def __init__(self, probs, precision="fp64", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("WaveHoltzBatch needs a CUDA device (libewh.so has no CPU path)")
        self.torch = torch
        self.probs = list(probs)
        self._keep = []
        items = []
        for p in self.probs:
            if getattr(p, "mapping", None) is not None:
                raise ValueError("batch members must be Cartesian grids (mapped grids run as WaveHoltz contexts)")
            desc = make_desc(p.dim, p.n, p.h, p.order, p.bc, PRECISIONS[precision], p.cfl, p.periods,
                             p.corrected, 0, getattr(p, "implicit", 0))
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.rho, p.lam, p.mu, p.forcing)]
            self._keep.append(arrs)
            items.append((desc, arrs[0], arrs[1], arrs[2], p.omega, arrs[3], p.nrhs))
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.b = L.ewh_batch_create(items, s)
        self._keep = None
        self.infos = [L.ewh_get_info(L.ewh_batch_member(self.b, k)) for k in range(len(self.probs))]
        self.sizes = [int(i.n_unknowns) * p.nrhs for i, p in zip(self.infos, self.probs)]

    def _vecs(self, xs=None):
        t = self.torch
        if xs is None:
            return [t.empty(n, dtype=t.float64, device="cuda") for n in self.sizes]
        out = []
        for x in xs:
            if not isinstance(x, t.Tensor):
                x = t.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
            out.append(x.to(device="cuda", dtype=t.float64).contiguous().reshape(-1))
        return out

    def apply_S(self, vs):
        vin = self._vecs(vs)
        vout = self._vecs()
        L.ewh_batch_apply_S(self.b, vin, vout)
        return vout

    def apply_Pi0(self):
        """b = Pi 0 of every member (each member context's own apply)."""
        out = self._vecs()
        for k, o in enumerate(out):
            L.ewh_apply_Pi0(L.ewh_batch_member(self.b, k), o)
        return out

    def solve(self, tol=1e-8, maxit=100000, raise_on_error=True):
        out = self._vecs()
        infos = L.ewh_batch_solve(self.b, tol, maxit, out, raise_on_error=raise_on_error)
        return out, infos

    def kernel_launches(self):
        return L.ewh_batch_kernel_launches(self.b)

    def close(self):
        if getattr(self, "b", None) is not None:
            self.torch.cuda.synchronize()
            L.ewh_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
