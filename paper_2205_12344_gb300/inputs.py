"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only *generates problem data* (grids, media, forcing, random
vectors).  It holds none of the method's arithmetic: no difference operators,
no time stepping, no filter.  Both the CUDA path and the oracle receive the
arrays produced here.

Conventions (the problem statement of Section 2.1: rho u_tt = div T(u) - f cos(wt),
T(u) = lambda (div u) I + 2 mu D(u); Dirichlet u = 0 or traction free T(u)n = 0):

* A grid has ``n[a]`` nodes along axis a *including* its two boundary nodes,
  spacing ``h``; node i of axis a sits at ``i * h``.
* ``bc`` lists the condition of the sides (x-, x+, y-, y+, z-, z+):
  0 = Dirichlet (boundary nodes fixed to zero, not unknowns),
  1 = free surface (boundary nodes are unknowns).
* Media (rho, lambda, mu) and forcing are sampled at every node of the full
  grid, C order ``[z][y][x]`` (x fastest); forcing is ``[rhs][comp][z][y][x]``.
* Vectors the solver works on hold unknown nodes only, ``[rhs][comp][z][y][x]``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

DIRICHLET = 0
FREE = 1


@dataclasses.dataclass
class Problem:
    """A complete synthetic problem: grid, medium, frequency and forcing."""

    name: str
    dim: int
    n: List[int]            # full-grid nodes per axis (x, y[, z])
    h: float
    order: int
    bc: List[int]           # 6 entries
    omega: float
    rho: np.ndarray         # full grid, shape n[::-1]
    lam: np.ndarray
    mu: np.ndarray
    forcing: np.ndarray     # [nrhs][dim][full grid]
    cfl: float = 0.5
    periods: int = 1
    corrected: int = 1
    implicit: int = 0       # 1: implicit time stepping (needs an explicit nt >= 5)
    mapping: Optional[Tuple[np.ndarray, np.ndarray]] = None  # (x, y) node coordinates: mapped 2D grid

    @property
    def nrhs(self) -> int:
        return int(self.forcing.shape[0])

    def unknowns_per_axis(self) -> List[int]:
        out = []
        for a in range(self.dim):
            k = self.n[a]
            k -= 1 if self.bc[2 * a] == DIRICHLET else 0
            k -= 1 if self.bc[2 * a + 1] == DIRICHLET else 0
            out.append(k)
        return out

    def n_nodes(self) -> int:
        return int(np.prod(self.unknowns_per_axis()))

    def n_unknowns(self) -> int:
        """Unknowns of one right-hand side (all components)."""
        return self.dim * self.n_nodes()


def _coords(n: Sequence[int], h: float):
    """Node coordinates, arrays broadcast to the full grid shape (z, y, x)."""
    axes = [np.arange(k, dtype=np.float64) * h for k in n]
    if len(n) == 2:
        y, x = np.meshgrid(axes[1], axes[0], indexing="ij")
        return [x, y]
    z, y, x = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return [x, y, z]


def full_shape(n: Sequence[int]):
    return tuple(int(k) for k in n[::-1])


# ----------------------------------------------------------------------------
# Media
# ----------------------------------------------------------------------------

def homogeneous(n, rho=1.0, lam=2.0, mu=1.0):
    s = full_shape(n)
    return (np.full(s, rho), np.full(s, lam), np.full(s, mu))


def layered(n, h, n_layers=8, vp=(1.5, 4.5), rho=(1.8, 2.6), depth_axis=1,
            top_is_high=True):
    """Horizontal layers of equal thickness; Vp and rho rise linearly with depth.

    Vs = Vp / sqrt(3) (so lambda = mu); mu = rho Vs^2, lambda = rho Vp^2 - 2 mu.
    Units: km, km/s, g/cc.  The free surface is the high end of ``depth_axis``;
    depth is measured from there.
    """
    s = full_shape(n)
    L = (n[depth_axis] - 1) * h
    coord = _coords(n, h)[depth_axis]
    depth = (L - coord) if top_is_high else coord
    k = np.minimum((depth / L * n_layers).astype(np.int64), n_layers - 1)
    t = k / max(n_layers - 1, 1)
    vp_l = vp[0] + (vp[1] - vp[0]) * t
    rho_l = rho[0] + (rho[1] - rho[0]) * t
    vs_l = vp_l / math.sqrt(3.0)
    mu = rho_l * vs_l ** 2
    lam = rho_l * vp_l ** 2 - 2.0 * mu
    return (np.broadcast_to(rho_l, s).copy(), np.broadcast_to(lam, s).copy(),
            np.broadcast_to(mu, s).copy())


def gaussian_random_field(n, h, corr=0.1, std=0.2, seed=0):
    """Zero-mean stationary field with Gaussian covariance exp(-r^2/(2 corr^2)).

    White noise filtered in Fourier space (periodic on a grid padded by
    3 correlation lengths so the wrap-around does not show), then scaled to
    the exact sample standard deviation ``std``.
    """
    rng = np.random.default_rng(seed)
    pad = int(math.ceil(3 * corr / h))
    shp = tuple(k + pad for k in full_shape(n))
    noise = rng.standard_normal(shp)
    spec = np.fft.rfftn(noise)
    freqs = [np.fft.fftfreq(k, d=h) for k in shp[:-1]] + [np.fft.rfftfreq(shp[-1], d=h)]
    grids = np.meshgrid(*freqs, indexing="ij")
    k2 = sum((2 * np.pi * g) ** 2 for g in grids)
    spec *= np.exp(-0.25 * k2 * corr ** 2)
    field = np.fft.irfftn(spec, s=shp)
    sl = tuple(slice(0, k) for k in full_shape(n))
    field = field[sl]
    field = field - field.mean()
    field *= std / field.std()
    return field


def grf_medium(n, h, seed=0, corr=0.1, std=0.2, vp_over_vs=1.8, rho=1.0, vs0=1.0):
    """log Vs = GRF(std, corr); Vp = vp_over_vs * Vs; constant rho."""
    logvs = gaussian_random_field(n, h, corr=corr, std=std, seed=seed)
    vs = vs0 * np.exp(logvs)
    vp = vp_over_vs * vs
    r = np.full(vs.shape, rho)
    mu = r * vs ** 2
    lam = r * vp ** 2 - 2 * mu
    return r, lam, mu


# ----------------------------------------------------------------------------
# Forcing
# ----------------------------------------------------------------------------

def gaussian_source(n, h, center, sigma, direction):
    """f(x) = direction * exp(-|x - center|^2 / (2 sigma^2)), shape [dim][grid]."""
    xs = _coords(n, h)
    r2 = sum((x - c) ** 2 for x, c in zip(xs, center))
    g = np.exp(-r2 / (2 * sigma ** 2))
    return np.stack([d * g for d in direction])


def ricker_source(n, h, center, s, direction):
    """Ricker-shaped (Mexican hat) spatial profile (1 - r^2/s^2) exp(-r^2/(2 s^2))."""
    xs = _coords(n, h)
    r2 = sum((x - c) ** 2 for x, c in zip(xs, center))
    g = (1.0 - r2 / s ** 2) * np.exp(-r2 / (2 * s ** 2))
    return np.stack([d * g for d in direction])


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def cfg_homogeneous_2d(nu=64, omega=10.0, order=2, bc=None, nrhs=1):
    """2D unit square, Dirichlet, rho=1, lambda=2, mu=1, Gaussian x-source
    (sigma 0.05, centre (0.4, 0.5)); ``nu`` unknowns per side, h = 1/(nu+1)."""
    bc = list(bc) if bc is not None else [DIRICHLET] * 4 + [DIRICHLET] * 2
    n = [nu + 2, nu + 2]
    h = 1.0 / (nu + 1)
    rho, lam, mu = homogeneous(n)
    f = gaussian_source(n, h, (0.4, 0.5), 0.05, (1.0, 0.0))
    forcing = np.stack([f] * nrhs)
    return Problem("homogeneous2d_%d" % nu, 2, n, h, order, bc, omega, rho, lam, mu, forcing)


def cfg_layered_2d(nu=1024, order=4, nrhs=1, shot_x=None, ppw=10.0, omega_scale=1.0):
    """2D layered medium: ``nu`` unknowns in x, ``nu`` + free top row in depth,
    h = 10 m, free top / Dirichlet elsewhere, Ricker vertical source at 5% depth.
    omega gives ``ppw`` points per shear wavelength in the slowest layer."""
    h = 0.01
    n = [nu + 2, nu + 2]          # x: Dirichlet both; y: Dirichlet bottom, free top
    bc = [DIRICHLET, DIRICHLET, DIRICHLET, FREE, DIRICHLET, DIRICHLET]
    rho, lam, mu = layered(n, h)
    vs_min = 1.5 / math.sqrt(3.0)
    omega = omega_scale * 2 * math.pi * vs_min / (ppw * h)
    L = (n[0] - 1) * h
    depth = 0.05 * (n[1] - 1) * h
    ytop = (n[1] - 1) * h
    s = ppw * h / 4.0
    if shot_x is None:
        shot_x = [0.5 * L] * nrhs
    forcing = np.stack([ricker_source(n, h, (sx, ytop - depth), s, (0.0, 1.0)) for sx in shot_x])
    return Problem("layered2d_%d" % nu, 2, n, h, order, bc, omega, rho, lam, mu, forcing)


def cfg_grf_3d(nu=256, order=4, seed=0, ppw=10.0):
    """3D unit cube, Dirichlet, log Vs Gaussian random field (std 0.2, corr 0.1),
    Vp = 1.8 Vs, rho = 1, point-Gaussian source (sigma 2h) at the centre along
    (1,1,1)/sqrt(3); omega gives ``ppw`` points per wavelength at min Vs."""
    n = [nu + 2] * 3
    h = 1.0 / (nu + 1)
    rho, lam, mu = grf_medium(n, h, seed=seed)
    vs_min = float(np.sqrt(mu / rho).min())
    omega = 2 * math.pi * vs_min / (ppw * h)
    d = 1.0 / math.sqrt(3.0)
    f = gaussian_source(n, h, (0.5, 0.5, 0.5), 2 * h, (d, d, d))
    return Problem("grf3d_%d" % nu, 3, n, h, order, [DIRICHLET] * 6, omega, rho, lam, mu, f[None])


def cfg_grf_2d(nu=256, order=2, seed=0, omega_scale=1.0, src=(0.5, 0.5), ppw=10.0):
    """2D unit square GRF medium (warm-start family): Dirichlet, Gaussian source."""
    n = [nu + 2, nu + 2]
    h = 1.0 / (nu + 1)
    rho, lam, mu = grf_medium(n, h, seed=seed)
    vs_min = float(np.sqrt(mu / rho).min())
    omega = omega_scale * 2 * math.pi * vs_min / (ppw * h)
    f = gaussian_source(n, h, src, 2 * h, (1.0, 0.0))
    return Problem("grf2d_%d" % nu, 2, n, h, order, [DIRICHLET] * 6, omega, rho, lam, mu, f[None])


def random_medium(n, seed, lam_range=(0.5, 3.0), mu_range=(0.5, 2.0), rho_range=(0.8, 1.5)):
    """Rough i.i.d. media for small parity/invariant tests."""
    rng = np.random.default_rng(seed)
    s = full_shape(n)
    return (rng.uniform(*rho_range, s), rng.uniform(*lam_range, s), rng.uniform(*mu_range, s))


def small_problem(dim, nu, order, bc, seed=0, nrhs=1, omega=None, h=None):
    """Tiny problem on an arbitrary grid (``nu`` unknown-ish nodes per axis) with a
    rough random medium and random smooth-ish forcing: for parity/edge tests."""
    rng = np.random.default_rng(1000 + seed)
    nu = list(nu) if isinstance(nu, (list, tuple)) else [nu] * dim
    n = [k + 2 for k in nu]
    h = h if h is not None else 1.0 / (max(n) - 1)
    rho, lam, mu = random_medium(n, seed)
    forcing = rng.standard_normal((nrhs, dim) + full_shape(n))
    if omega is None:
        omega = 2.3 + 0.37 * seed + (max(n) - 1) * 0.35
    return Problem("small%dd" % dim, dim, n, h, order, list(bc) + [0] * (6 - len(bc)),
                   float(omega), rho, lam, mu, forcing)


def annulus_mapping(n, h, span=math.pi / 3, r0=1.0, dr=0.5):
    """Node coordinates (x, y), each of full_shape(n), of an annular sector: the
    radius r0 + dr q' along q and the angle span r' along r (q', r' in [0, 1]
    over the grid), so the mapping preserves orientation.  The sector's extent
    is set by r0, dr and span alone; h is taken for the common (n, h)
    signature of the mapping generators."""
    q = np.arange(n[0]) / (n[0] - 1)
    r = np.arange(n[1]) / (n[1] - 1)
    Q, R = np.meshgrid(q, r)
    rad = r0 + dr * Q
    ang = span * R
    return rad * np.cos(ang), rad * np.sin(ang)


def wavy_mapping(n, h, amp=0.04):
    """Node coordinates of a smoothly skewed, non-orthogonal square: x = q +
    amp L sin(2 pi r / L) + (amp L / 2) sin(pi q / L) sin(pi r / L),
    y = r + amp L sin(2 pi q / L), L the side length (n - 1) h per axis."""
    Lq, Lr = (n[0] - 1) * h, (n[1] - 1) * h
    Q, R = np.meshgrid(np.arange(n[0]) * h, np.arange(n[1]) * h)
    X = Q + amp * Lq * np.sin(2 * np.pi * R / Lr) + 0.5 * amp * Lq * np.sin(np.pi * Q / Lq) * np.sin(np.pi * R / Lr)
    Y = R + amp * Lr * np.sin(2 * np.pi * Q / Lq)
    return X, Y


def random_vectors(prob: Problem, count: int, seed: int) -> np.ndarray:
    """``count`` random unknown-vectors (float64), shape [count][nrhs*dim*nodes]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, prob.nrhs * prob.n_unknowns()))


def unknown_index(prob: Problem) -> np.ndarray:
    """Full-grid array (z, y, x) holding each node's index among the unknown
    nodes of one component, or -1 for a Dirichlet boundary node."""
    shape = full_shape(prob.n)
    known = np.ones(shape, dtype=bool)
    for a in range(prob.dim):
        ax = prob.dim - 1 - a                    # numpy axis of grid axis a
        sl_lo = [slice(None)] * prob.dim
        sl_hi = [slice(None)] * prob.dim
        sl_lo[ax] = 0
        sl_hi[ax] = -1
        if prob.bc[2 * a] == DIRICHLET:
            known[tuple(sl_lo)] = False
        if prob.bc[2 * a + 1] == DIRICHLET:
            known[tuple(sl_hi)] = False
    idx = np.full(shape, -1, dtype=np.int64)
    idx[known] = np.arange(int(known.sum()))
    return idx


def window_problem(prob: Problem, lo: Sequence[int], hi: Sequence[int]) -> Problem:
    """Crop ``prob`` to full-grid nodes lo[a]..hi[a] (inclusive) per axis.

    Sides of the window that are not sides of the domain become Dirichlet
    (their boundary layer is held at zero).  Used to evaluate single entries
    of a large S apply inside their domain of dependence.  A mapped problem
    keeps the node coordinates of the window.
    """
    sl = tuple(slice(lo[a], hi[a] + 1) for a in reversed(range(prob.dim)))
    bc = list(prob.bc)
    for a in range(prob.dim):
        if lo[a] > 0:
            bc[2 * a] = DIRICHLET
        if hi[a] < prob.n[a] - 1:
            bc[2 * a + 1] = DIRICHLET
    n = [hi[a] - lo[a] + 1 for a in range(prob.dim)]
    fsl = (slice(None), slice(None)) + sl
    return Problem(prob.name + "_win", prob.dim, n, prob.h, prob.order, bc, prob.omega,
                   prob.rho[sl].copy(), prob.lam[sl].copy(), prob.mu[sl].copy(),
                   prob.forcing[fsl].copy(), cfl=prob.cfl, periods=prob.periods,
                   corrected=prob.corrected, implicit=getattr(prob, "implicit", 0),
                   mapping=None if getattr(prob, "mapping", None) is None
                   else (prob.mapping[0][sl].copy(), prob.mapping[1][sl].copy()))
