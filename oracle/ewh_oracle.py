"""Plain FP64 CPU oracle of the El-WaveHoltz hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import this module.  The product path never calls it; it
shares no code with the CUDA library (no kernels, tables or helpers).

What it computes, in the paper's order and notation:

* Section 2.1: rho u_tt = div T(u) - f cos(w t), T(u) = lambda (div u) I + 2 mu D(u),
  Dirichlet (u = 0) or traction-free (T(u) n = 0) sides: energy conserving.
* Section 4.1, eq. (symmertic_FD): M (u^{n+1} - 2u^n + u^{n-1}) = dt^2 L_h u^n with
  L_h symmetric and M diagonal (scaled by 1/2 on free sides, 1/4 at free
  corners).  The paper leaves the Cartesian L_h to its reference; the reading
  used here is the Hessian of a discrete elastic energy E(u) = 1/2 u^T K u,
  L_h = -K (assembled term by term below, see ``assemble``).
* Section 4.3, eq. (elastic-time-explicit-corrected): dt^2 is replaced by
  (w~^2 / w^2) dt^2 with w~ = 2 sin(w dt / 2) / dt, and u^{-1} is the Taylor
  start u^0 + (k/2) M^{-1} (L_h u^0 - W f) (the printed start is garbled; this
  is the start that makes v cos(w t_n) an exact discrete solution).
* Section 3, eq. (el_WHI_OP), with the trapezoidal rule of Section 4 and
  eq. (qoper): Pi u0 = sum_n w_n u^n, w_n = (2/N) eta_n (cos(w t_n) - 1/4);
  S = Pi with f = 0; eq. (many_periods_filter) for K periods.
* Section 4.5, eq. (amat_sym): CG on M (I - S) v = M Pi 0 (conjugate residual as
  in the Section 4.5 remark; MINRES as in the Section 4.4 remark on indefinite
  systems).
* Section 4.4: the implicit (corrected) scheme, each level a sparse solve.
* Section 4.1, curvilinear form: mapped 2D grids (order 4), ``assemble_mapped``.
* Appendix B: the discrete filter transfer function beta_h.

Parity is pinned by tests/test_oracle_*.py against closed forms, invariants,
a sparse direct solve of the discrete Helmholtz problem and manufactured
solutions (see those files).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DIRICHLET = 0
FREE = 1


# ----------------------------------------------------------------------------
# One-axis building blocks on the full node line 0..N-1 (both ends boundary nodes)
# ----------------------------------------------------------------------------

def edge_difference(N):
    """(N-1) x N: (Delta u)_{i+1/2} = u_{i+1} - u_i."""
    return sp.diags([-np.ones(N - 1), np.ones(N - 1)], [0, 1], shape=(N - 1, N), format="csr")


def edge_average(N):
    """(N-1) x N: edge value = mean of the two end nodes."""
    return sp.diags([0.5 * np.ones(N - 1), 0.5 * np.ones(N - 1)], [0, 1], shape=(N - 1, N), format="csr")


def centred_difference(N):
    """N x N first difference at nodes: (u_{i+1} - u_{i-1}) / 2 inside, the
    one-sided u_1 - u_0 and u_{N-1} - u_{N-2} at the two ends (used only where
    the end is a free surface; Dirichlet ends carry zero nodal weight)."""
    C = sp.lil_matrix((N, N))
    for i in range(1, N - 1):
        C[i, i - 1] = -0.5
        C[i, i + 1] = 0.5
    C[0, 0], C[0, 1] = -1.0, 1.0
    C[N - 1, N - 2], C[N - 1, N - 1] = -1.0, 1.0
    return C.tocsr()


def axis_weight(N, lo, hi):
    """Trapezoid factor of each node along one axis: 1/2 on a free end."""
    m = np.ones(N)
    if lo == FREE:
        m[0] = 0.5
    if hi == FREE:
        m[-1] = 0.5
    return m


def axis_unknown(N, lo, hi):
    """True where the node is an unknown (Dirichlet ends are fixed to zero)."""
    k = np.ones(N, dtype=bool)
    if lo == DIRICHLET:
        k[0] = False
    if hi == DIRICHLET:
        k[-1] = False
    return k


def _along(axis, op, n):
    """Lift a 1D operator acting on ``axis`` to the full grid (C order z,y,x)."""
    dim = len(n)
    mats = []
    for a in reversed(range(dim)):          # slowest axis first
        mats.append(op if a == axis else sp.identity(n[a], format="csr"))
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def _outer(vecs):
    """Tensor product of per-axis vectors (x first) flattened in C order z,y,x."""
    out = np.ones(1)
    for v in reversed(vecs):
        out = np.kron(out, v)
    return out


# ----------------------------------------------------------------------------
# Spatial operator: K = -L_h and the mass M (reading of Section 4.1)
# ----------------------------------------------------------------------------

@dataclass
class System:
    dim: int
    n: list
    h: float
    order: int
    bc: list
    omega: float
    K: sp.csr_matrix = None          # unknowns x unknowns (one rhs, all comps)
    Mdiag: np.ndarray = None         # rho * m * h^d per unknown
    Wdiag: np.ndarray = None         # m * h^d per unknown
    rho_u: np.ndarray = None         # rho per unknown
    sel: np.ndarray = None           # flat full-grid indices of unknown nodes
    f_over_rho: np.ndarray = None    # [nrhs][unknowns]  M^{-1} W f
    f_u: np.ndarray = None           # [nrhs][unknowns]  f at unknowns
    nt: int = 0                      # time steps per period
    periods: int = 1
    dt: float = 0.0
    kt: float = 0.0                  # c dt^2
    c: float = 1.0
    omega_tilde: float = 0.0
    weights: np.ndarray = None       # trapezoid filter weights, length periods*nt+1
    corrected: int = 1
    implicit: int = 0                # 1: the implicit scheme of Section 4.4
    alpha: float = 2.0               # its centre coefficient (eq. alpha; 2 when uncorrected)
    impl_lu: object = None           # factorisation of M + (dt^2/2) K (implicit scheme)


def sbp4_first_derivative(N):
    """Fourth-order diagonal-norm summation-by-parts first derivative on the
    node line 0..N-1 (unit spacing) and its norm H.

    Inside: (u_{i-2} - 8 u_{i-1} + 8 u_{i+1} - u_{i+2}) / 12.  The first and
    last four rows use the classical closure of the diagonal-norm 2-4 operator,
    H = diag(17/48, 59/48, 43/48, 49/48, 1, ...), so that H D + (H D)^T =
    diag(-1, 0, ..., 0, 1) (pinned in the tests together with its accuracy).
    """
    if N < 8:
        raise ValueError("order 4 needs at least 8 nodes per axis")
    Hb = [17.0 / 48, 59.0 / 48, 43.0 / 48, 49.0 / 48]
    Db = [[-24.0 / 17, 59.0 / 34, -4.0 / 17, -3.0 / 34, 0.0, 0.0],
          [-0.5, 0.0, 0.5, 0.0, 0.0, 0.0],
          [4.0 / 43, -59.0 / 86, 0.0, 59.0 / 86, -4.0 / 43, 0.0],
          [3.0 / 98, 0.0, -59.0 / 98, 0.0, 32.0 / 49, -4.0 / 49]]
    D = sp.lil_matrix((N, N))
    H = np.ones(N)
    for i in range(4, N - 4):
        D[i, i - 2], D[i, i - 1], D[i, i + 1], D[i, i + 2] = 1.0 / 12, -8.0 / 12, 8.0 / 12, -1.0 / 12
    for i in range(4):
        H[i] = H[N - 1 - i] = Hb[i]
        for j in range(6):
            if Db[i][j] != 0.0:
                D[i, j] = Db[i][j]
                D[N - 1 - i, N - 1 - j] = -Db[i][j]
    return D.tocsr(), H


def assemble(dim, n, h, order, bc, rho, lam, mu):
    """Assemble K (= -L_h) and the diagonal mass M on the unknowns.

    K is the Hessian of a discrete elastic energy E(u) = 1/2 u^T K u that
    approximates 1/2 int lambda (div u)^2 + 2 mu D(u):D(u) (Section 2.1);
    Dirichlet nodes enter with value zero and are then dropped, free sides get
    the natural (traction-free) condition.  The whole form scales by h^(d-2),
    M = rho * m * h^d.

    order 2 (compact):
      E = 1/2 sum_{a, alpha} sum_{edges e along a} w_e C^{alpha a}_e (Delta_a u_alpha)_e^2
        + sum_{a<b} sum_nodes m [ lambda (C_a u_a)(C_b u_b) + mu (C_b u_a)(C_a u_b) ]
      C^{alpha a} = lambda + 2 mu if alpha == a else mu, edge value = mean of the
      two end nodes; m = product over axes of the trapezoid factor (1/2 on a
      free side), zero on Dirichlet nodes; w_e = that product over the axes
      other than a; C_a = centred first difference, one-sided on free boundary
      nodes.  Inside, this is the classical 9-point (2D) conservative stencil.

    order 4 (summation by parts):
      E = 1/2 sum_nodes H [ lambda (sum_a D_a u_a)^2 + 2 mu sum_{a,b} eps_ab^2 ],
      eps_ab = (D_b u_a + D_a u_b) / 2, D_a = ``sbp4_first_derivative`` along a,
      H = product of the per-axis SBP norms (also the mass weights).
    """
    if order not in (2, 4):
        raise ValueError("order must be 2 or 4")
    nn = int(np.prod(n))
    lam_f = lam.reshape(-1)
    mu_f = mu.reshape(-1)
    axk = [axis_unknown(n[a], bc[2 * a], bc[2 * a + 1]) for a in range(dim)]
    known = _outer([k.astype(float) for k in axk]) > 0.5
    blocks = [[None] * dim for _ in range(dim)]

    if order == 2:
        P_f = lam_f + 2.0 * mu_f
        axw = [axis_weight(n[a], bc[2 * a], bc[2 * a + 1]) for a in range(dim)]
        m_node = _outer(axw) * known
        weight = _outer(axw)
        D = [_along(a, edge_difference(n[a]), n) for a in range(dim)]
        A = [_along(a, edge_average(n[a]), n) for a in range(dim)]
        C = [_along(a, centred_difference(n[a]), n) for a in range(dim)]
        w_edge = []
        for a in range(dim):
            vecs = [np.ones(n[a] - 1) if b == a else axw[b] for b in range(dim)]
            w_edge.append(_outer(vecs))
        for al in range(dim):
            Kaa = sp.csr_matrix((nn, nn))
            for a in range(dim):
                coef = P_f if al == a else mu_f
                Kaa = Kaa + D[a].T @ sp.diags(w_edge[a] * (A[a] @ coef)) @ D[a]
            blocks[al][al] = Kaa
        for a in range(dim):
            for b in range(a + 1, dim):
                Kab = C[a].T @ sp.diags(m_node * lam_f) @ C[b] + C[b].T @ sp.diags(m_node * mu_f) @ C[a]
                blocks[a][b] = Kab
                blocks[b][a] = Kab.T
    else:
        Ds, Hs = [], []
        for a in range(dim):
            d1, h1 = sbp4_first_derivative(n[a])
            Ds.append(_along(a, d1, n))
            Hs.append(h1)
        weight = _outer(Hs)
        HL = sp.diags(weight * lam_f)
        HM = sp.diags(weight * mu_f)
        # d E / d u_alpha = sum_b D_b^T H sigma_{alpha b},
        # sigma_{alpha b} = lambda delta_{alpha b} div u + mu (D_b u_alpha + D_alpha u_b)
        for al in range(dim):
            for be in range(dim):
                Kab = Ds[al].T @ HL @ Ds[be] + Ds[be].T @ HM @ Ds[al]
                if al == be:
                    for b in range(dim):
                        Kab = Kab + Ds[b].T @ HM @ Ds[b]
                blocks[al][be] = Kab

    Kfull = sp.bmat(blocks, format="csr") * (h ** (dim - 2))
    sel = np.nonzero(known)[0]
    sel_all = np.concatenate([sel + c * nn for c in range(dim)])
    K = Kfull[sel_all][:, sel_all].tocsr()
    rho_f = rho.reshape(-1)
    Mdiag = np.tile(rho_f[sel] * weight[sel] * h ** dim, dim)
    Wdiag = np.tile(weight[sel] * h ** dim, dim)
    rho_u = np.tile(rho_f[sel], dim)
    return K, Mdiag, Wdiag, rho_u, sel


def mapped_metrics(n, h, X, Y):
    """Metric terms of a smooth mapping x(q, r), y(q, r) sampled on the node
    grid (q, r) = (i h, j h) (Section 4.1, curvilinear form): x_q, x_r, y_q,
    y_r from the fourth-order SBP derivative, J = x_q y_r - x_r y_q and
    q_x = y_r / J, q_y = -x_r / J, r_x = -y_q / J, r_y = x_q / J (flattened,
    C order y, x).  Returns (J, qx, qy, rx, ry)."""
    Dq = _along(0, sbp4_first_derivative(n[0])[0], n) / h
    Dr = _along(1, sbp4_first_derivative(n[1])[0], n) / h
    x, y = X.reshape(-1), Y.reshape(-1)
    xq, xr, yq, yr = Dq @ x, Dr @ x, Dq @ y, Dr @ y
    J = xq * yr - xr * yq
    return J, yr / J, -xr / J, -yq / J, xq / J


def assemble_mapped(n, h, bc, rho, lam, mu, X, Y):
    """K (= -L_h) and M on the unknowns for a 2D curvilinear grid, order 4
    (Section 4.1, curvilinear form; the energy reading of the Cartesian case
    carried over): the energy density 1/2 [lambda (div u)^2 + 2 mu eps:eps]
    with physical derivatives d/dx = q_x d/dq + r_x d/dr, d/dy = q_y d/dq +
    r_y d/dr (SBP D in q and r), summed with the weight H J h^2; the mass is
    rho J H h^2 (the paper's rho J).  With X = q, Y = r it is the Cartesian
    order-4 operator."""
    dim = 2
    nn = int(np.prod(n))
    J, qx, qy, rx, ry = mapped_metrics(n, h, X, Y)
    d0, h0 = sbp4_first_derivative(n[0])
    d1, h1 = sbp4_first_derivative(n[1])
    Dq = _along(0, d0, n) / h
    Dr = _along(1, d1, n) / h
    Dx = sp.diags(qx) @ Dq + sp.diags(rx) @ Dr
    Dy = sp.diags(qy) @ Dq + sp.diags(ry) @ Dr
    Ds = [Dx.tocsr(), Dy.tocsr()]
    weight = _outer([h0, h1])
    wJ = weight * J * h ** 2
    HL = sp.diags(wJ * lam.reshape(-1))
    HM = sp.diags(wJ * mu.reshape(-1))
    blocks = [[None] * dim for _ in range(dim)]
    for al in range(dim):
        for be in range(dim):
            Kab = Ds[al].T @ HL @ Ds[be] + Ds[be].T @ HM @ Ds[al]
            if al == be:
                for b in range(dim):
                    Kab = Kab + Ds[b].T @ HM @ Ds[b]
            blocks[al][be] = Kab
    Kfull = sp.bmat(blocks, format="csr")
    axk = [axis_unknown(n[a], bc[2 * a], bc[2 * a + 1]) for a in range(dim)]
    known = _outer([k.astype(float) for k in axk]) > 0.5
    sel = np.nonzero(known)[0]
    sel_all = np.concatenate([sel + c * nn for c in range(dim)])
    K = Kfull[sel_all][:, sel_all].tocsr()
    rho_f = rho.reshape(-1)
    Mdiag = np.tile(rho_f[sel] * wJ[sel], dim)
    Wdiag = np.tile(wJ[sel], dim)
    rho_u = np.tile(rho_f[sel], dim)
    return K, Mdiag, Wdiag, rho_u, sel


def cfl_dt_mapped(n, h, cfl, rho, lam, mu, X, Y):
    """Time-step bound on a mapped grid: dt = cfl h / sqrt(max over nodes of
    (lambda + 3 mu)/rho * (|grad q|^2 + |grad r|^2) / 2); the Cartesian bound
    when the mapping is the identity."""
    J, qx, qy, rx, ry = mapped_metrics(n, h, X, Y)
    s2 = (qx * qx + qy * qy + rx * rx + ry * ry) / 2.0
    c2 = ((lam + 3 * mu) / rho).reshape(-1)
    return cfl * h / math.sqrt(np.max(c2 * s2))


def cfl_dt(dim, order, h, cfl, rho, lam, mu):
    """Time-step bound dt_CFL = cfl * h / sqrt(max over nodes of (lambda + (d+1) mu) / rho).

    Both spatial orders keep h^2 * rho(M^{-1} K) below 4 max((lambda+(d+1)mu)/rho),
    so the leapfrog (stable while c dt^2 rho(M^{-1}K) < 4) is stable for cfl < 1."""
    speed2 = np.max((lam + (dim + 1) * mu) / rho)
    return cfl * h / math.sqrt(speed2)


def filter_weights(nt, periods):
    """Trapezoid weights of eq. (many_periods_filter) over K = periods periods:
    w_n = 2/(K nt) * eta_n * (cos(2 pi n / nt) - 1/4), eta = 1/2 at both ends."""
    N = nt * periods
    nvec = np.arange(N + 1)
    eta = np.ones(N + 1)
    eta[0] = eta[-1] = 0.5
    return (2.0 / N) * eta * (np.cos(2.0 * np.pi * nvec / nt) - 0.25)


def build_system(prob, nt: Optional[int] = None) -> System:
    """Medium + grid + forcing -> System (reading of Sections 2.1, 4.1, 4.3)."""
    dim, n, h, order = prob.dim, list(prob.n), prob.h, prob.order
    bc = list(prob.bc)
    mapping = getattr(prob, "mapping", None)
    if mapping is not None:
        if dim != 2 or order != 4:
            raise ValueError("mapped grids: 2D, order 4")
        K, Mdiag, Wdiag, rho_u, sel = assemble_mapped(n, h, bc, prob.rho, prob.lam, prob.mu, *mapping)
    else:
        K, Mdiag, Wdiag, rho_u, sel = assemble(dim, n, h, order, bc, prob.rho, prob.lam, prob.mu)
    s = System(dim=dim, n=n, h=h, order=order, bc=bc, omega=prob.omega)
    s.K, s.Mdiag, s.Wdiag, s.rho_u, s.sel = K, Mdiag, Wdiag, rho_u, sel
    nn = int(np.prod(n))
    f = prob.forcing.reshape(prob.forcing.shape[0], dim, nn)[:, :, sel].reshape(prob.forcing.shape[0], -1)
    s.f_u = f
    s.f_over_rho = f / rho_u[None, :]
    T = 2.0 * math.pi / prob.omega
    if nt is None:
        dtc = (cfl_dt_mapped(n, h, prob.cfl, prob.rho, prob.lam, prob.mu, *mapping) if mapping is not None
               else cfl_dt(dim, order, h, prob.cfl, prob.rho, prob.lam, prob.mu))
        nt = max(5, int(math.ceil(T / dtc)))
    s.nt = nt
    s.periods = prob.periods
    s.dt = T / nt
    s.omega_tilde = 2.0 * math.sin(prob.omega * s.dt / 2.0) / s.dt
    s.corrected = prob.corrected
    s.c = (s.omega_tilde / prob.omega) ** 2 if prob.corrected else 1.0
    s.kt = s.c * s.dt ** 2
    s.weights = filter_weights(nt, prob.periods)
    if getattr(prob, "implicit", 0):
        # Section 4.4: (u^{n+1} - alpha u^n + u^{n-1}) / dt^2 = (1/2) L_h (u^{n+1} + u^{n-1})
        #              - f cos(w t_n) cos(w dt),  alpha = cos(w dt) (2 + w^2 dt^2) (eq. alpha)
        s.implicit = 1
        wd = prob.omega * s.dt
        s.alpha = math.cos(wd) * (2.0 + wd * wd) if prob.corrected else 2.0
        s.omega_tilde = 2.0 * math.sin(wd / 2.0) / (s.dt * math.sqrt(math.cos(wd))) if math.cos(wd) > 0 else float("nan")
        s.kt = 0.0
    return s


# ----------------------------------------------------------------------------
# Time stepping and the WaveHoltz operator (Sections 3, 4.3, eq. qoper)
# ----------------------------------------------------------------------------

def minv_K(s: System, u):
    """M^{-1} K u (= -M^{-1} L_h u) for one right-hand side."""
    return (s.K @ u) / s.Mdiag


def apply_Pi_implicit(s: System, u0, rhs: int = 0, forced: bool = True):
    """Pi u0 / S u0 with the implicit scheme of Section 4.4, in the mass form
    (M + (dt^2/2) K) u^{n+1} = alpha M u^n - (M + (dt^2/2) K) u^{n-1}
                                - dt^2 W f cos(w t_n) cos(w dt),
    started from (M + (dt^2/2) K) u^{-1} = (alpha/2) M u0 - (dt^2/2) W f cos(w dt)
    (the paper's modified initial data), with the trapezoidal filter
    accumulation of eq. (qoper).  Each level is a sparse direct solve."""
    dt = s.dt
    c = 0.5 * dt * dt
    if s.impl_lu is None:
        s.impl_lu = spla.splu((sp.diags(s.Mdiag) + c * s.K).tocsc())
    lu = s.impl_lu
    cdt = math.cos(s.omega * dt)
    wf = s.Wdiag * s.f_u[rhs] if forced else np.zeros_like(u0)

    def B(u):
        return s.Mdiag * u + c * (s.K @ u)

    u_prev = lu.solve(s.Mdiag * (0.5 * s.alpha * u0) - c * wf * cdt)
    u = u0.copy()
    acc = s.weights[0] * u
    N = s.nt * s.periods
    for n in range(N):
        cos_n = math.cos(2.0 * math.pi * n / s.nt)
        u_next = lu.solve(s.alpha * (s.Mdiag * u) - B(u_prev) - dt * dt * wf * cos_n * cdt)
        u_prev, u = u, u_next
        acc = acc + s.weights[n + 1] * u
    return acc


def apply_Pi(s: System, u0, rhs: int = 0, forced: bool = True, return_history=False):
    """Pi u0 (forced) or S u0 (forced=False): corrected leapfrog over
    periods*nt steps with the trapezoidal filter accumulation (the implicit
    scheme when the system was built with it)."""
    if s.implicit:
        assert not return_history
        return apply_Pi_implicit(s, u0, rhs, forced)
    kt = s.kt
    N = s.nt * s.periods
    g = s.f_over_rho[rhs] if forced else np.zeros_like(u0)
    u_prev = u0 + 0.5 * kt * (-minv_K(s, u0) - g)          # u^{-1}
    u = u0.copy()
    acc = s.weights[0] * u
    hist = [u.copy()] if return_history else None
    for n in range(N):
        cos_n = math.cos(2.0 * math.pi * n / s.nt)
        u_next = 2.0 * u - u_prev + kt * (-minv_K(s, u) - g * cos_n)
        u_prev, u = u, u_next
        acc = acc + s.weights[n + 1] * u
        if return_history:
            hist.append(u.copy())
    if return_history:
        return acc, hist
    return acc


def apply_S(s: System, v, rhs: int = 0):
    return apply_Pi(s, v, rhs=rhs, forced=False)


def apply_Pi0(s: System, rhs: int = 0):
    return apply_Pi(s, np.zeros(s.K.shape[0]), rhs=rhs, forced=True)


def discrete_energy(s: System, u_now, u_next):
    """Eq. (8) generalised to k = c dt^2: ||u^{n+1}-u^n||_M^2 / k + (u^{n+1})^T K u^n."""
    d = u_next - u_now
    return float(d @ (s.Mdiag * d)) / s.kt + float(u_next @ (s.K @ u_now))


def leapfrog_energy_history(s: System, u0, steps):
    """Unforced leapfrog from (u0, u_t = 0) for ``steps`` steps; energy per step."""
    kt = s.kt
    u_prev = u0 + 0.5 * kt * (-minv_K(s, u0))
    u = u0.copy()
    out = []
    for _ in range(steps):
        u_next = 2.0 * u - u_prev + kt * (-minv_K(s, u))
        out.append(discrete_energy(s, u, u_next))
        u_prev, u = u, u_next
    return np.array(out)


# ----------------------------------------------------------------------------
# Krylov solve of M (I - S) v = M b (eq. amat_sym) and the direct definition
# ----------------------------------------------------------------------------

@dataclass
class SolveInfo:
    iters: int = 0
    rel_res: float = float("nan")
    converged: bool = False
    history: list = field(default_factory=list)


def mdot(s: System, x, y):
    """The M inner product of eq. (amat_sym), sum_i x_i M_i y_i, rounded once
    (math.fsum of the products x_i M_i y_i): the value does not depend on the
    order of summation, so any split of the vectors reproduces it exactly."""
    return math.fsum(x * s.Mdiag * y)


def cg_solve(s: System, tol=1e-8, maxit=10000, x0=None, rhs: int = 0, b=None):
    """CG in the M inner product on (I - S) v = b, b = Pi 0.  Stops when
    ||b - (I - S) x||_M / ||b||_M <= tol (recursive residual)."""
    if b is None:
        b = apply_Pi0(s, rhs)
    bb = math.sqrt(mdot(s, b, b))
    info = SolveInfo()
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - (x - apply_S(s, x, rhs))
    p = r.copy()
    rr = mdot(s, r, r)
    info.history.append(math.sqrt(rr) / bb)
    if math.sqrt(rr) / bb <= tol:
        info.converged = True
        info.rel_res = math.sqrt(rr) / bb
        return x, info
    for it in range(1, maxit + 1):
        q = p - apply_S(s, p, rhs)
        pq = mdot(s, p, q)
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = mdot(s, r, r)
        info.history.append(math.sqrt(rr_new) / bb)
        info.iters = it
        if math.sqrt(rr_new) / bb <= tol:
            info.converged = True
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    info.rel_res = info.history[-1]
    return x, info


def cr_solve(s: System, tol=1e-8, maxit=10000, x0=None, rhs: int = 0, b=None):
    """Conjugate residual in the M inner product on (I - S) v = b (Section 4.5
    remark: the residual norm does not increase).  One S apply per iteration."""
    if b is None:
        b = apply_Pi0(s, rhs)

    def A(v):
        return v - apply_S(s, v, rhs)

    bb = math.sqrt(mdot(s, b, b))
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    info.history.append(math.sqrt(mdot(s, r, r)) / bb)
    if info.history[-1] <= tol:
        info.converged, info.rel_res = True, info.history[-1]
        return x, info
    Ar = A(r)
    p, Ap = r.copy(), Ar.copy()
    rAr = mdot(s, r, Ar)
    for it in range(1, maxit + 1):
        alpha = rAr / mdot(s, Ap, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        info.history.append(math.sqrt(mdot(s, r, r)) / bb)
        info.iters = it
        if info.history[-1] <= tol:
            info.converged = True
            break
        Ar = A(r)
        rAr_new = mdot(s, r, Ar)
        beta = rAr_new / rAr
        rAr = rAr_new
        p = r + beta * p
        Ap = Ar + beta * Ap
    info.rel_res = info.history[-1]
    return x, info


def minres(apply_A, b, mw, tol=1e-8, maxit=10000, x0=None):
    """MINRES for a system A x = b whose A is self-adjoint in the inner
    product (x, y)_W = sum mw x y (Section 4.4, the remark on the implicit
    scheme: when few quadrature points make beta_h exceed 1 near a resonance
    the system may be indefinite, and MINRES replaces CG).

    Lanczos in the W inner product builds the tridiagonal T_k; its QR
    factorisation by Givens rotations gives the iterate minimising the
    W-norm of the residual over x0 + K_k, updated by the direction recurrence
    w_k = (v_k - rho2 w_{k-1} - rho3 w_{k-2}) / rho1.  The residual norm is the
    last rotated right-hand side entry.  Returns x, SolveInfo (history of
    ||r||_W / ||b||_W)."""
    def dot(x, y):
        return float(np.dot(mw * x, y))

    bb = math.sqrt(dot(b, b))
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    beta = math.sqrt(dot(r, r))
    info.history.append(beta / bb)
    if info.history[-1] <= tol:
        info.converged, info.rel_res = True, info.history[-1]
        return x, info
    v_prev = np.zeros_like(b)
    v = r / beta
    w1 = np.zeros_like(b)   # w_{k-1}
    w2 = np.zeros_like(b)   # w_{k-2}
    c1, s1 = 1.0, 0.0       # rotation k-1
    c2, s2 = 1.0, 0.0       # rotation k-2
    eta = beta
    for it in range(1, maxit + 1):
        # Lanczos step: A v_k = beta_k v_{k-1} + alpha_k v_k + beta_{k+1} v_{k+1}
        z = apply_A(v) - beta * v_prev
        alpha = dot(v, z)
        z = z - alpha * v
        beta_next = math.sqrt(max(dot(z, z), 0.0))
        # the previous two rotations act on the new column (0, beta_k, alpha_k, beta_{k+1})
        rho3 = s2 * beta
        t = c2 * beta
        rho2 = c1 * t + s1 * alpha
        delta = -s1 * t + c1 * alpha
        rho1 = math.hypot(delta, beta_next)
        if rho1 == 0.0:
            raise ZeroDivisionError("MINRES: singular tridiagonal")
        c, sn = delta / rho1, beta_next / rho1
        w = (v - rho2 * w1 - rho3 * w2) / rho1
        x = x + (c * eta) * w
        eta = -sn * eta
        info.history.append(abs(eta) / bb)
        info.iters = it
        if info.history[-1] <= tol or beta_next == 0.0:
            info.converged = info.history[-1] <= tol or beta_next == 0.0
            break
        w2, w1 = w1, w
        c2, s2, c1, s1 = c1, s1, c, sn
        v_prev, v = v, z / beta_next
        beta = beta_next
    info.rel_res = info.history[-1]
    return x, info


def minres_solve(s: System, tol=1e-8, maxit=10000, x0=None, rhs: int = 0, b=None):
    """MINRES on (I - S) v = b in the M inner product (one S apply per iteration)."""
    if b is None:
        b = apply_Pi0(s, rhs)
    return minres(lambda v: v - apply_S(s, v, rhs), b, s.Mdiag, tol=tol, maxit=maxit, x0=x0)


def helmholtz_direct(s: System, rhs: int = 0):
    """Definition-level solution: (w_eff^2 M - K) v = W f with w_eff = w for
    the corrected scheme and w~ for the standard one (Section 4.3)."""
    w = s.omega if s.corrected else s.omega_tilde
    A = (w * w) * sp.diags(s.Mdiag) - s.K
    return spla.spsolve(A.tocsc(), s.Wdiag * s.f_u[rhs])


def form_S(s: System):
    """S as a dense matrix, column by column (tiny grids only)."""
    N = s.K.shape[0]
    S = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0.0
        e[j] = 1.0
        S[:, j] = apply_S(s, e)
    return S


# ----------------------------------------------------------------------------
# Filter transfer functions (Section 3 and Appendix B)
# ----------------------------------------------------------------------------

def beta_continuous(lam_over_omega):
    """beta(r w) = (1/pi) int_0^{2 pi} (cos t - 1/4) cos(r t) dt in closed form:
    (1/pi) [ (sin 2pi(1-r))/(2(1-r)) + (sin 2pi(1+r))/(2(1+r)) - (sin 2pi r)/(4 r) ],
    each quotient sin(2 pi x)/x taken as its limit 2 pi at x = 0."""
    r = np.atleast_1d(np.asarray(lam_over_omega, dtype=np.float64))

    def sinc2pi(x):
        out = np.full_like(x, 2.0 * np.pi)
        nz = np.abs(x) > 1e-14
        out[nz] = np.sin(2.0 * np.pi * x[nz]) / x[nz]
        return out

    return (0.5 * sinc2pi(1.0 - r) + 0.5 * sinc2pi(1.0 + r) - 0.25 * sinc2pi(r)) / np.pi


def beta_h(r, M):
    """App. B: beta_h(r) = (dt/pi) sum_{n=0}^M eta_n cos(r t_n) (cos t_n - 1/4),
    t_n = n dt, dt = 2 pi / M."""
    dt = 2.0 * np.pi / M
    t = np.arange(M + 1) * dt
    eta = np.ones(M + 1)
    eta[0] = eta[-1] = 0.5
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return (dt / np.pi) * (np.cos(np.outer(r, t)) @ (eta * (np.cos(t) - 0.25)))


def leftmost_unit_crossing(M, lo=0.5, hi=1.0, iters=200):
    """Bisection for the leftmost r* < 1 with beta_h(r*) = 1 (App. B)."""
    # beta_h < 1 well below resonance; scan for the first point with beta_h >= 1
    grid = np.linspace(lo, hi, 20001)
    vals = beta_h(grid, M) - 1.0
    idx = int(np.argmax(vals >= 0.0))
    a, b = grid[idx - 1], grid[idx]
    for _ in range(iters):
        mid = 0.5 * (a + b)
        if beta_h(mid, M)[0] - 1.0 >= 0.0:
            b = mid
        else:
            a = mid
    return 0.5 * (a + b)
