"""Multi-rank layouts of the hot path.

Independent systems per rank: the WaveHoltz solves of different shots and
frequencies are independent problems, so they shard across ranks with no
data-path collective.  Only the bookkeeping is collective: the slowest rank's
time and the total work.  This is what the GPU benchmark runs.

One system split into slabs (``Slab``, ``slab_wave_solve``, ``slab_cg``):
the layout of a solve too large for one device.  Following the paper's
account of the method's communication (Section 1: the wave solves need only
local exchanges between neighbours at every time step, and the global inner
products come once per period; Section 3: once per K periods with the
many-periods filter), the unknown planes along the slowest grid axis are
split into contiguous slabs; each rank keeps a halo of ``halo`` planes on
each cut side, advances ``halo // reach`` leapfrog levels between exchanges
(the valid region shrinks by the operator's plane reach per level), and the
CG inner products are exactly rounded sums gathered from every rank, so the
result does not depend on the split.  The spatial operator on a rank's
extended region is supplied by the caller; every machine this runs on gives
a process one GPU, so these ranks are CPU processes (gloo).
"""
from __future__ import annotations

import math
from typing import Callable, List, Sequence

import numpy as np


def shard(n_items: int, rank: int, world: int) -> List[int]:
    """Round-robin assignment of item indices to ``rank`` of ``world``."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must lie in [0, world)")
    return list(range(rank, n_items, world))


def shot_positions(length: float, n_shots: int) -> List[float]:
    """Evenly spaced shot positions strictly inside [0, length]."""
    return [length * (k + 1) / (n_shots + 1) for k in range(n_shots)]


def reduce_job(elapsed_s: float, work_units: float, device=None):
    """(max elapsed over ranks, total work over ranks); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_s, work_units
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def gather_results(local: Sequence, n_items: int, rank: int, world: int):
    """Reassemble per-item results computed by ``shard`` on every rank into
    item order (every rank receives the full list)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or world == 1:
        return list(local)
    parts = [None] * world
    dist.all_gather_object(parts, list(local))
    out = [None] * n_items
    for r in range(world):
        for k, idx in enumerate(shard(n_items, r, world)):
            out[idx] = parts[r][k]
    return out


# ----------------------------------------------------------------------------
# One system split into slabs
# ----------------------------------------------------------------------------

def slab_ranges(n_planes: int, world: int):
    """Contiguous, balanced [lo, hi) plane ranges of ``world`` ranks."""
    if world < 1 or n_planes < world:
        raise ValueError("need at least one plane per rank")
    base, extra = divmod(n_planes, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


class Slab:
    """Rank ``rank``'s slab of a vector laid out [comp][plane][rest]: ``dim``
    components of ``n_planes`` planes of ``plane_size`` unknowns each (the
    planes run along the slowest axis of the unknown grid).  The rank owns
    planes [lo, hi) and keeps ``halo`` more planes on each cut side
    ([elo, ehi)); every slab must be at least ``halo`` planes thick, so a
    halo comes from the neighbouring rank alone."""

    def __init__(self, dim: int, n_planes: int, plane_size: int, world: int, rank: int, halo: int):
        self.dim, self.n_planes, self.plane_size = dim, n_planes, plane_size
        self.world, self.rank, self.halo = world, rank, halo
        self.ranges = slab_ranges(n_planes, world)
        if min(hi - lo for lo, hi in self.ranges) < halo and world > 1:
            raise ValueError("every slab must be at least `halo` planes thick")
        self.lo, self.hi = self.ranges[rank]
        self.elo = max(0, self.lo - halo)
        self.ehi = min(n_planes, self.hi + halo)

    # index sets (into the global vector of one right-hand side)
    def _planes(self, a, b):
        per = self.n_planes * self.plane_size
        return np.concatenate([np.arange(c * per + a * self.plane_size, c * per + b * self.plane_size)
                               for c in range(self.dim)])

    def own_global(self):
        return self._planes(self.lo, self.hi)

    def ext_global(self):
        return self._planes(self.elo, self.ehi)

    def own_in_ext(self):
        """Positions of the owned entries inside the extended local vector."""
        ext = (self.ehi - self.elo) * self.plane_size
        a = (self.lo - self.elo) * self.plane_size
        b = (self.hi - self.elo) * self.plane_size
        return np.concatenate([np.arange(c * ext + a, c * ext + b) for c in range(self.dim)])

    def _view(self, v_ext):
        return v_ext.reshape(self.dim, self.ehi - self.elo, self.plane_size)

    def exchange(self, *arrays):
        """Refresh the halo planes of extended local vectors from the
        neighbours' owned planes (torch.distributed point-to-point; the
        owned planes of every array must be valid)."""
        if self.world == 1:
            return
        import torch
        import torch.distributed as dist
        ops, recvs = [], []
        for v in arrays:
            w = self._view(v)
            if self.rank > 0:            # lower neighbour: my planes [lo, lo + halo) are its upper halo
                send = torch.from_numpy(np.ascontiguousarray(w[:, self.lo - self.elo:self.lo - self.elo + self.halo]))
                buf = torch.empty((self.dim, self.lo - self.elo, self.plane_size), dtype=torch.float64)
                ops.append(dist.P2POp(dist.isend, send, self.rank - 1))
                ops.append(dist.P2POp(dist.irecv, buf, self.rank - 1))
                recvs.append((w, slice(0, self.lo - self.elo), buf))
            if self.rank < self.world - 1:  # upper neighbour: my planes [hi - halo, hi) are its lower halo
                a = self.hi - self.elo
                send = torch.from_numpy(np.ascontiguousarray(w[:, a - self.halo:a]))
                buf = torch.empty((self.dim, self.ehi - self.hi, self.plane_size), dtype=torch.float64)
                ops.append(dist.P2POp(dist.isend, send, self.rank + 1))
                ops.append(dist.P2POp(dist.irecv, buf, self.rank + 1))
                recvs.append((w, slice(a, self.ehi - self.elo), buf))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for w, sl, buf in recvs:
            w[:, sl] = buf.numpy()


def slab_wave_solve(slab: Slab, minv_K_ext: Callable, u0_own, g_ext, nt: int, periods: int, kt: float,
                    weights, reach: int):
    """The filtered wave solve of one right-hand side on a slab: Pi u0 over
    nt * periods levels of the time-corrected leapfrog with the Taylor start
    (Section 4.3) and the trapezoid accumulation (eq. qoper); S u0 when
    ``g_ext`` is zero.  ``minv_K_ext`` maps an extended local vector to
    M^{-1} K of it, exact on every plane whose stencil lies in the extended
    region; ``reach`` is the operator's reach in planes.  Halos are exchanged
    whenever another level would leave the owned planes invalid.  Returns
    the accumulator on the owned planes."""
    if slab.world > 1 and slab.halo < reach:
        raise ValueError("the halo must cover at least one operator reach")
    own = slab.own_in_ext()
    u = np.zeros(slab.dim * (slab.ehi - slab.elo) * slab.plane_size)
    u[own] = u0_own
    slab.exchange(u)
    u_prev = u + 0.5 * kt * (-minv_K_ext(u) - g_ext)
    big = 1 << 30                                   # no cut side: always valid
    H = slab.halo if slab.world > 1 else big
    vu, vp = H, H - reach                          # valid planes beyond the owned ones
    acc = weights[0] * u[own]
    for n in range(nt * periods):
        if min(vu - reach, vp) < 0:
            slab.exchange(u, u_prev)
            vu = vp = H
        cos_n = math.cos(2.0 * math.pi * n / nt)
        u_next = 2.0 * u - u_prev + kt * (-minv_K_ext(u) - g_ext * cos_n)
        u_prev, u = u, u_next
        vp, vu = vu, min(vu - reach, vp)
        acc = acc + weights[n + 1] * u[own]
    return acc


def exact_partials(values):
    """Non-overlapping partial sums whose exact sum is the exact sum of
    ``values`` (Shewchuk's summation, J. R. Shewchuk, Adaptive precision
    floating-point arithmetic, 1997): a rank's exact contribution to a sum
    that is rounded once at the end."""
    partials: List[float] = []
    for x in values:
        i = 0
        for y in partials:
            if abs(x) < abs(y):
                x, y = y, x
            hi = x + y
            lo = y - (hi - x)
            if lo:
                partials[i] = lo
                i += 1
            x = hi
        partials[i:] = [x]
    return partials


def slab_mdot(x_own, y_own, m_own, world: int = 1):
    """The M inner product sum x_i M_i y_i over every rank's owned entries,
    rounded once: each rank's exact partial sums are gathered and summed by
    math.fsum, so the value is the same for any split (and equals the
    exactly rounded sum of the undivided vectors)."""
    parts = exact_partials((x_own * m_own * y_own).tolist())
    if world > 1:
        import torch.distributed as dist
        allp = [None] * world
        dist.all_gather_object(allp, parts)
        parts = [v for p in allp for v in p]
    return math.fsum(parts)


def slab_cg(apply_S_own: Callable, b_own, m_own, world: int, tol: float = 1e-8, maxit: int = 10000):
    """CG in the M inner product on (I - S) v = b (Section 4.5, eq.
    amat_sym) over slabs: the vectors stay distributed, S is applied by
    ``apply_S_own`` (a ``slab_wave_solve``), and each iteration gathers the
    two inner products (p, (I - S)p)_M and (r, r)_M.  Stops when
    ||r||_M / ||b||_M <= tol (recursive residual).  Returns (x_own, history
    of relative residuals)."""
    bb = math.sqrt(slab_mdot(b_own, b_own, m_own, world))
    x = np.zeros_like(b_own)
    r = b_own.copy()
    p = r.copy()
    rr = slab_mdot(r, r, m_own, world)
    hist = [math.sqrt(rr) / bb]
    if hist[-1] <= tol:
        return x, hist
    for _ in range(maxit):
        q = p - apply_S_own(p)
        pq = slab_mdot(p, q, m_own, world)
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = slab_mdot(r, r, m_own, world)
        hist.append(math.sqrt(rr_new) / bb)
        if hist[-1] <= tol:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, hist
