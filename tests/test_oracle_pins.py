"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself: the references are closed forms, library routines used as an
independent second computation (scipy quadrature, dense eigensolvers, sparse
direct solves), textbook stencils, manufactured solutions and numbers printed
in the paper (tests/golden/).
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.sparse.linalg as spla

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------- filter (Section 3, App. B)

@pytest.mark.parametrize("nt", [5, 7, 50, 183])
@pytest.mark.parametrize("periods", [1, 2, 3])
def test_filter_weight_identities(nt, periods):
    """Trapezoid weights reproduce beta(0) = -1/2 and the fixed-point identity
    sum_n w_n cos(w t_n) = 1 (Section 3; eq. many_periods_filter)."""
    w = O.filter_weights(nt, periods)
    t = 2 * np.pi * np.arange(nt * periods + 1) / nt
    g = _golden_kv("section3_filter.txt")
    assert w.shape == (nt * periods + 1,)
    assert abs(w.sum() - g["beta_at_0"]) < 1e-13
    assert abs((w * np.cos(t)).sum() - g["beta_at_omega"]) < 1e-13


def test_beta_closed_form_against_quadrature():
    """beta(lambda) of Section 3 in closed form vs scipy adaptive quadrature."""
    r = np.array([0.0, 0.3, 0.999, 1.0, 1.001, 1.7, 2.0, 5.25])
    closed = O.beta_continuous(r)
    for ri, bi in zip(r, closed):
        q, _ = si.quad(lambda t: (math.cos(t) - 0.25) * math.cos(ri * t), 0, 2 * math.pi,
                       epsabs=1e-14, epsrel=1e-14, limit=200)
        assert abs(bi - q / math.pi) < 1e-12
    g = _golden_kv("section3_filter.txt")
    assert abs(closed[0] - g["beta_at_0"]) < 1e-15
    assert abs(closed[3] - g["beta_at_omega"]) < 1e-15


def test_beta_h_tends_to_beta():
    """App. B: the trapezoid beta_h approximates beta with O(dt^2) error."""
    r = np.linspace(0.0, 3.0, 31)
    e = [np.abs(O.beta_h(r, M) - O.beta_continuous(r)).max() for M in (40, 80, 160)]
    assert e[1] < e[0] / 3.5 and e[2] < e[1] / 3.5


def test_appendix_b_gap_bound():
    """App. B: 1 - r* <= 0.022 dt^2 for M = 5..100 quadrature points."""
    g = _golden_kv("appendix_b_gap.txt")
    for M in range(int(g["m_min"]), int(g["m_max"]) + 1):
        rs = O.leftmost_unit_crossing(M)
        dt = 2 * np.pi / M
        assert rs < 1.0
        assert 1.0 - rs <= g["coefficient"] * dt * dt, (M, 1 - rs, g["coefficient"] * dt * dt)
        # the bound is not vacuous: the gap is within a factor 3 of it
        assert 1.0 - rs > g["coefficient"] * dt * dt / 3.0


# ---------------------------------------------------------------- SBP operator (order 4)

def test_sbp4_summation_by_parts_and_accuracy():
    """H D + (H D)^T = diag(-1, 0, ..., 0, 1); boundary rows exact for
    quadratics, interior rows for quartics."""
    N = 20
    D, H = O.sbp4_first_derivative(N)
    Q = np.diag(H) @ D.toarray()
    B = np.zeros((N, N))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.abs(Q + Q.T - B).max() < 1e-14
    x = np.arange(N, dtype=float)
    for p in range(5):
        err = D @ x ** p - (p * x ** (p - 1) if p else 0 * x)
        if p <= 2:
            assert np.abs(err).max() < 1e-11
        assert np.abs(err[4:-4]).max() < 1e-9 * max(1, N ** p)
    assert abs(H.sum() - (N - 1)) < 1e-13          # the norm integrates constants exactly


# ---------------------------------------------------------------- spatial operator (Section 4.1)

def _bc_list(dim):
    sides = 2 * dim
    for bc in itertools.product([O.DIRICHLET, O.FREE], repeat=sides):
        yield list(bc) + [0] * (6 - sides)


@pytest.mark.parametrize("order", [2, 4])
def test_stiffness_symmetric_positive_definite_2d(order):
    """L_h symmetric and negative definite when a side is Dirichlet (Section 4.1)."""
    for bc in _bc_list(2):
        if all(b == O.FREE for b in bc[:4]):
            continue
        for seed in range(2):
            p = inputs.small_problem(2, [7, 8], order, bc, seed=seed)
            K, Md, *_ = O.assemble(2, p.n, p.h, order, p.bc, p.rho, p.lam, p.mu)
            Kd = K.toarray()
            assert np.abs(Kd - Kd.T).max() <= 1e-13 * np.abs(Kd).max()
            ev = np.linalg.eigvalsh(Kd)
            assert ev[0] > 1e-6 * ev[-1], (bc, ev[0], ev[-1])


@pytest.mark.parametrize("order", [2, 4])
def test_stiffness_spd_3d(order):
    for bc in ([0] * 6, [0, 0, 0, 0, 0, 1], [1, 0, 0, 1, 0, 1]):
        p = inputs.small_problem(3, [6, 7, 6], order, bc, seed=3)
        K, Md, *_ = O.assemble(3, p.n, p.h, order, p.bc, p.rho, p.lam, p.mu)
        Kd = K.toarray()
        assert np.abs(Kd - Kd.T).max() <= 1e-13 * np.abs(Kd).max()
        ev = np.linalg.eigvalsh(Kd)
        assert ev[0] > 1e-6 * ev[-1]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_body_modes_have_zero_energy(order, dim):
    """With every side free, translations and infinitesimal rotations carry no
    elastic energy (D(u) = 0): a dropped or mis-signed mixed term breaks this."""
    nu = [7, 8] if dim == 2 else [6, 7, 6]
    p = inputs.small_problem(dim, nu, order, [O.FREE] * (2 * dim), seed=5)
    K, Md, Wd, rho, sel = O.assemble(dim, p.n, p.h, order, p.bc, p.rho, p.lam, p.mu)
    xs = inputs._coords(p.n, p.h)
    pts = [x.reshape(-1)[sel] for x in xs]
    nn = len(sel)
    modes = []
    for a in range(dim):                         # translations
        m = np.zeros(dim * nn)
        m[a * nn:(a + 1) * nn] = 1.0
        modes.append(m)
    for a, b in itertools.combinations(range(dim), 2):   # rotations in the (a,b) plane
        m = np.zeros(dim * nn)
        m[a * nn:(a + 1) * nn] = -pts[b]
        m[b * nn:(b + 1) * nn] = pts[a]
        modes.append(m)
    scale = abs(K).max()
    for m in modes:
        assert np.abs(K @ m).max() < 1e-12 * scale * max(1.0, np.abs(m).max())
    # and a shear is not a zero mode
    m = np.zeros(dim * nn)
    m[:nn] = pts[1]
    m[nn:2 * nn] = pts[0]
    assert np.abs(K @ m).max() > 1e-3 * scale * p.h


def test_order2_interior_matches_textbook_stencil():
    """Homogeneous medium, order 2: the interior row of -K/h^2 equals the
    classical second-order operator (lambda+2mu) u_xx + mu u_yy + (lambda+mu) v_xy
    with the 4-point mixed difference (u_{i+1,j+1} - u_{i+1,j-1} - u_{i-1,j+1} + u_{i-1,j-1})/4h^2."""
    lam, mu = 2.0, 1.0
    nu = 9
    p = inputs.cfg_homogeneous_2d(nu=nu)
    p.lam[:] = lam
    p.mu[:] = mu
    K, Md, *_ = O.assemble(2, p.n, p.h, 2, p.bc, p.rho, p.lam, p.mu)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(2 * nu * nu)
    lhs = -(K @ u)               # h^(d-2) = 1 in 2D; textbook uses raw differences
    U = u[:nu * nu].reshape(nu, nu)
    V = u[nu * nu:].reshape(nu, nu)
    Up = np.pad(U, 1)
    Vp = np.pad(V, 1)
    c = slice(1, -1)
    uxx = Up[c, 2:] - 2 * Up[c, c] + Up[c, :-2]
    uyy = Up[2:, c] - 2 * Up[c, c] + Up[:-2, c]
    vxx = Vp[c, 2:] - 2 * Vp[c, c] + Vp[c, :-2]
    vyy = Vp[2:, c] - 2 * Vp[c, c] + Vp[:-2, c]
    vxy = (Vp[2:, 2:] - Vp[:-2, 2:] - Vp[2:, :-2] + Vp[:-2, :-2]) / 4
    uxy = (Up[2:, 2:] - Up[:-2, 2:] - Up[2:, :-2] + Up[:-2, :-2]) / 4
    ref_u = (lam + 2 * mu) * uxx + mu * uyy + (lam + mu) * vxy
    ref_v = mu * vxx + (lam + 2 * mu) * vyy + (lam + mu) * uxy
    got_u = lhs[:nu * nu].reshape(nu, nu)
    got_v = lhs[nu * nu:].reshape(nu, nu)
    assert np.abs(got_u - ref_u).max() < 1e-12
    assert np.abs(got_v - ref_v).max() < 1e-12


def test_order4_interior_matches_composed_fourth_order_differences():
    """Homogeneous medium, order 4: far from the sides, -K/h^2 applies the
    fourth-order centred difference twice (wide stencil):
    (lambda+2mu) c4(c4 u)_xx + mu (c4 c4 u)_yy + (lambda+mu) c4_x c4_y v."""
    lam, mu = 2.0, 1.0
    nu = 20
    p = inputs.cfg_homogeneous_2d(nu=nu, order=4)
    K, Md, *_ = O.assemble(2, p.n, p.h, 4, p.bc, p.rho, p.lam, p.mu)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(2 * nu * nu)
    H = (Md[:nu * nu] / p.h ** 2).reshape(nu, nu)   # interior weights are 1
    lhs_u = (-(K @ u)[:nu * nu]).reshape(nu, nu)
    lhs_v = (-(K @ u)[nu * nu:]).reshape(nu, nu)
    U = u[:nu * nu].reshape(nu, nu)
    V = u[nu * nu:].reshape(nu, nu)

    def cx(A):
        return (A[:, :-4] - 8 * A[:, 1:-3] + 8 * A[:, 3:-1] - A[:, 4:]) / 12

    def cy(A):
        return (A[:-4, :] - 8 * A[1:-3, :] + 8 * A[3:-1, :] - A[4:, :]) / 12

    ref_u = (lam + 2 * mu) * cx(cx(U))[4:-4, :] + mu * cy(cy(U))[:, 4:-4] + (lam + mu) * cx(cy(V))[2:-2, 2:-2]
    ref_v = mu * cx(cx(V))[4:-4, :] + (lam + 2 * mu) * cy(cy(V))[:, 4:-4] + (lam + mu) * cx(cy(U))[2:-2, 2:-2]
    # unknown j is grid node j+1; the SBP closure touches grid nodes 0..5
    got = (lhs_u / H)[6:-6, 6:-6]
    want = ref_u[2:-2, 2:-2]
    assert got.shape == want.shape
    assert np.abs(got - want).max() < 1e-11
    gotv = (lhs_v / H)[6:-6, 6:-6]
    wantv = ref_v[2:-2, 2:-2]
    assert np.abs(gotv - wantv).max() < 1e-11


# ---------------------------------------------------------------- manufactured solutions

def _mms_error(order, bc, ns, uv, coef, omega=1.3, corrected=1):
    """Max-norm error of the discrete Helmholtz solution (the El-WaveHoltz fixed
    point, Section 4.3) against a manufactured continuous solution of eq.
    (elastic-frequency) rho w^2 v + div T(v) = f."""
    sy = pytest.importorskip("sympy")
    X, Y = sy.symbols("x y")
    uex, vex = uv(sy, X, Y)
    lam, mu, rho = coef(sy, X, Y)
    ux, uy, vx, vy = sy.diff(uex, X), sy.diff(uex, Y), sy.diff(vex, X), sy.diff(vex, Y)
    sxx = lam * (ux + vy) + 2 * mu * ux
    syy = lam * (ux + vy) + 2 * mu * vy
    sxy = mu * (uy + vx)
    fx = rho * omega ** 2 * uex + sy.diff(sxx, X) + sy.diff(sxy, Y)
    fy = rho * omega ** 2 * vex + sy.diff(sxy, X) + sy.diff(syy, Y)
    fns = [sy.lambdify((X, Y), e, "numpy") for e in (fx, fy, uex, vex, lam, mu, rho)]
    errs = []
    for nu in ns:
        n = [nu + 2, nu + 2]
        h = 1.0 / (nu + 1)
        xs = np.arange(n[0]) * h
        Yg, Xg = np.meshgrid(xs, xs, indexing="ij")
        ev = [np.broadcast_to(np.asarray(f(Xg, Yg), dtype=float), Xg.shape).copy() for f in fns]
        prob = inputs.Problem("mms", 2, n, h, order, list(bc) + [0, 0], omega, ev[6], ev[4], ev[5],
                              np.stack([np.stack([ev[0], ev[1]])]), corrected=corrected)
        s = O.build_system(prob)
        vnum = O.helmholtz_direct(s)
        ex = np.concatenate([ev[2].reshape(-1)[s.sel], ev[3].reshape(-1)[s.sel]])
        errs.append(np.abs(vnum - ex).max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log((ns[i + 1] + 1) / (ns[i] + 1))
             for i in range(len(ns) - 1)]
    return errs, rates


def _sine(sy, X, Y):
    return sy.sin(sy.pi * X) * sy.sin(2 * sy.pi * Y), sy.sin(2 * sy.pi * X) * sy.sin(sy.pi * Y)


def _generic(sy, X, Y):
    return (X * (1 - X) * Y * (1 - Y) * sy.exp(X + Y / 2), sy.sin(sy.pi * X) * Y * (1 - Y) * (1 + X))


def _free_top(sy, X, Y):
    return (sy.sin(sy.pi * X) * Y * (1 - Y) ** 2 * (1 + Y), sy.sin(2 * sy.pi * X) * sy.sin(sy.pi * Y) * (1 - Y))


def _const(sy, X, Y):
    return 2, 1, 1


def _smooth(sy, X, Y):
    return 2 + sy.sin(X + Y), 1 + 0.3 * sy.cos(2 * X - Y), 1 + 0.2 * X * Y


@pytest.mark.parametrize("uv,coef,bc", [(_sine, _const, [0, 0, 0, 0]), (_sine, _smooth, [0, 0, 0, 0]),
                                        (_generic, _const, [0, 0, 0, 0]), (_free_top, _const, [0, 0, 0, 1])])
def test_mms_order2_rate(uv, coef, bc):
    errs, rates = _mms_error(2, bc, [15, 31, 63], uv, coef)
    assert 1.9 < rates[-1] < 2.15, (errs, rates)


@pytest.mark.parametrize("uv,coef,bc", [(_sine, _const, [0, 0, 0, 0]), (_sine, _smooth, [0, 0, 0, 0]),
                                        (_generic, _const, [0, 0, 0, 0]), (_free_top, _const, [0, 0, 0, 1])])
def test_mms_order4_rate(uv, coef, bc):
    """Order 4: fourth-order interior, second-order SBP boundary closure: the
    global error converges at (at least) third order."""
    errs, rates = _mms_error(4, bc, [15, 31, 63], uv, coef)
    assert rates[-1] > 2.7, (errs, rates)
    errs2, _ = _mms_error(2, bc, [63], uv, coef)
    assert errs[-1] < errs2[0]


def test_table1_quartic_rate():
    """Table 1: quartic solution, lambda = mu = 1, omega = 1, standard leapfrog,
    Dirichlet unit square: second-order convergence (paper rates 2.06/2.03/2.02)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_fd_errors.txt"))
            if l.strip() and not l.startswith("#")]
    paper_rates = [float(r[2]) for r in rows[1:]]
    ns = [int(r[0]) - 1 for r in rows[:3]]       # n points -> n-1 unknowns per side

    def quartic(sy, X, Y):
        q = 256 * X ** 2 * (X - 1) ** 2 * Y ** 2 * (Y - 1) ** 2
        return q, q

    def unit(sy, X, Y):
        return 1, 1, 1

    errs, rates = _mms_error(2, [0, 0, 0, 0], ns, quartic, unit, omega=1.0, corrected=0)
    for r, pr in zip(rates, paper_rates):
        assert abs(r - pr) < 0.12, (rates, paper_rates)
    # same order of magnitude as the printed errors
    assert 0.2 < errs[0] / float(rows[0][1]) < 5


# ---------------------------------------------------------------- time stepping (Section 4.3, eq. 8)

@pytest.mark.parametrize("dim,order,bc", [(2, 2, [0, 0, 0, 1]), (2, 4, [0, 0, 0, 1]), (2, 4, [1, 0, 1, 0]),
                                          (3, 2, [0, 0, 0, 0, 0, 1]), (3, 4, [0, 0, 0, 0, 1, 0])])
def test_discrete_energy_conserved(dim, order, bc):
    """Eq. (8): the unforced leapfrog conserves the discrete energy."""
    nu = [8, 9] if dim == 2 else [6, 7, 6]
    p = inputs.small_problem(dim, nu, order, bc, seed=4)
    s = O.build_system(p)
    u0 = np.random.default_rng(9).standard_normal(s.K.shape[0])
    e = O.leapfrog_energy_history(s, u0, 3000 if dim == 2 else 600)
    assert e.min() > 0
    assert (e.max() - e.min()) / e[0] < 1e-12


def test_cfl_bound_keeps_leapfrog_stable():
    """c dt^2 rho(M^{-1} K) < 4 at cfl 0.5 (and h^2 rho(M^{-1}K) <= 4 max((l+(d+1)m)/r))."""
    cases = [inputs.cfg_homogeneous_2d(nu=30, order=2), inputs.cfg_homogeneous_2d(nu=30, order=4),
             inputs.cfg_layered_2d(nu=40, order=4), inputs.cfg_layered_2d(nu=40, order=2),
             inputs.small_problem(3, [8, 8, 8], 4, [0, 0, 0, 0, 0, 1], seed=1),
             inputs.small_problem(3, [8, 8, 8], 2, [0, 0, 1, 0, 0, 1], seed=2)]
    for p in cases:
        s = O.build_system(p)
        Dm = 1.0 / np.sqrt(s.Mdiag)
        A = (s.K.multiply(Dm[:, None])).multiply(Dm[None, :]).tocsr()
        lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0]
        speed2 = np.max((p.lam + (p.dim + 1) * p.mu) / p.rho)
        assert lmax * p.h ** 2 <= 4.0 * speed2 * (1 + 1e-9), (p.name, lmax * p.h ** 2 / speed2)
        assert s.kt * lmax < 4.0 * 0.25 * 1.0001 + 1e-12     # cfl^2 * 4


# ---------------------------------------------------------------- WaveHoltz operator (Sections 3, 4.3, 4.5)

CASES = [(2, 2, [0, 0, 0, 0], 1), (2, 2, [0, 0, 0, 1], 1), (2, 4, [0, 0, 0, 1], 1),
         (2, 4, [1, 0, 0, 1], 2), (3, 2, [0, 0, 0, 0, 1, 0], 1), (3, 4, [0, 0, 0, 0, 0, 1], 1)]


def _case(dim, order, bc, periods, seed=7):
    nu = [8, 9] if dim == 2 else [6, 6, 7]
    p = inputs.small_problem(dim, nu, order, bc, seed=seed)
    p.periods = periods
    return p


@pytest.mark.parametrize("dim,order,bc,periods", CASES)
def test_fixed_point_is_discrete_helmholtz_solution(dim, order, bc, periods):
    """Sections 3 and 4.3: with the corrected scheme and the Taylor start, the
    solution of (w^2 M - K) v = W f is an exact fixed point of Pi_h."""
    s = O.build_system(_case(dim, order, bc, periods))
    v = O.helmholtz_direct(s)
    assert np.linalg.norm(O.apply_Pi(s, v) - v) <= 1e-12 * np.linalg.norm(v)


def test_uncorrected_scheme_converges_to_shifted_frequency():
    """Section 4.3: the standard leapfrog's fixed point solves the w~ problem,
    which differs from the w problem by O(dt^2)."""
    p = _case(2, 2, [0, 0, 0, 1], 1)
    p.corrected = 0
    s = O.build_system(p)
    v_tilde = O.helmholtz_direct(s)
    assert np.linalg.norm(O.apply_Pi(s, v_tilde) - v_tilde) <= 1e-12 * np.linalg.norm(v_tilde)
    p.corrected = 1
    s1 = O.build_system(p)
    v = O.helmholtz_direct(s1)
    assert np.linalg.norm(O.apply_Pi(s, v) - v) > 1e-6 * np.linalg.norm(v)


@pytest.mark.parametrize("dim,order,bc,periods", CASES)
def test_MA_symmetric_and_spectrum(dim, order, bc, periods):
    """Section 4.5, eq. (amat_sym): M(I - S) is symmetric; Section 3: the
    eigenvalues of A = I - S lie in (0, 3/2)."""
    s = O.build_system(_case(dim, order, bc, periods))
    S = O.form_S(s)
    A = np.eye(S.shape[0]) - S
    MA = s.Mdiag[:, None] * A
    assert np.abs(MA - MA.T).max() <= 1e-13 * np.abs(MA).max()
    ev = np.linalg.eigvalsh(0.5 * (MA + MA.T) / np.sqrt(s.Mdiag)[:, None] / np.sqrt(s.Mdiag)[None, :])
    g = _golden_kv("section3_filter.txt")
    assert ev.min() > g["A_eig_lower"] and ev.max() < g["A_eig_upper"]


@pytest.mark.parametrize("dim,order,bc,periods", CASES[:4])
def test_S_eigenvalues_follow_discrete_filter(dim, order, bc, periods):
    """Section 3 / App. B: S acts on each eigenmode of M^{-1}K (eigenvalue k2)
    by sum_n w_n cos(n theta), cos theta = 1 - c dt^2 k2 / 2."""
    s = O.build_system(_case(dim, order, bc, periods))
    Ms = np.sqrt(s.Mdiag)
    kap = np.linalg.eigvalsh(s.K.toarray() / Ms[:, None] / Ms[None, :])
    theta = np.arccos(1.0 - s.kt * kap / 2.0)
    nvec = np.arange(len(s.weights))
    pred = np.sort(np.cos(np.outer(theta, nvec)) @ s.weights)
    S = O.form_S(s)
    got = np.sort(np.linalg.eigvals(S).real)
    assert np.abs(pred - got).max() < 1e-11
    # and the same numbers from App. B's beta_h (K = 1: r = theta / (w dt))
    if periods == 1:
        r = theta / (s.omega * s.dt)
        assert np.abs(np.sort(O.beta_h(r, s.nt)) - pred).max() < 1e-12


@pytest.mark.parametrize("dim,order,bc,periods", CASES)
def test_cg_matches_direct_solve(dim, order, bc, periods):
    """Section 4.5: CG in the M inner product solves (I - S) v = Pi 0."""
    s = O.build_system(_case(dim, order, bc, periods))
    v = O.helmholtz_direct(s)
    x, info = O.cg_solve(s, tol=1e-12, maxit=500)
    assert info.converged
    assert np.linalg.norm(x - v) <= 1e-9 * np.linalg.norm(v)


def test_fixed_point_iteration_converges_slower_than_cg():
    """Section 3: u <- Pi u from u = 0 converges to the same v; CG is faster."""
    s = O.build_system(_case(2, 2, [0, 0, 0, 0], 1, seed=1))
    v = O.helmholtz_direct(s)
    u = np.zeros_like(v)
    for _ in range(400):
        u = O.apply_Pi(s, u)
    assert np.linalg.norm(u - v) < 1e-6 * np.linalg.norm(v)
    x, info = O.cg_solve(s, tol=1e-10)
    assert info.iters < 100


def test_more_periods_fewer_iterations():
    """Table 3 (qualitative): filtering over K periods lowers the iteration count."""
    p = inputs.cfg_homogeneous_2d(nu=20, omega=12.0)
    its = []
    for K in (1, 2, 3):
        p.periods = K
        s = O.build_system(p)
        x, info = O.cg_solve(s, tol=1e-8)
        its.append(info.iters)
    assert its[0] > its[1] > its[2], its


def test_windowed_S_equals_full_S_at_centre():
    """S v at one node depends only on v within (N_t + 2) r nodes: the oracle
    on a window around it gives the full-domain value (used for full-size
    sampled parity)."""
    p = inputs.cfg_layered_2d(nu=100, order=4)
    dtc = O.cfl_dt(2, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    p.omega = 2 * math.pi / (5.5 * dtc)               # N_t = 6: a window of radius 32 inside the grid
    s = O.build_system(p)
    assert s.nt == 6
    v = inputs.random_vectors(p, 1, 3)[0]
    full = O.apply_S(s, v)
    idx = inputs.unknown_index(p)
    r = 4                                             # order 4: D^T H D reaches 4 nodes per level
    R = (s.nt + 2) * r
    cx, cy = 50, 96                                   # near the free top
    lo = [max(0, cx - R), max(0, cy - R)]
    hi = [min(p.n[0] - 1, cx + R), min(p.n[1] - 1, cy + R)]
    assert lo[0] > 0 and hi[0] < p.n[0] - 1 and lo[1] > 0     # a true sub-window
    w = inputs.window_problem(p, lo, hi)
    sw = O.build_system(w, nt=s.nt)
    widx = inputs.unknown_index(w)
    nn, wnn = p.n_nodes(), w.n_nodes()
    vw = np.zeros(2 * wnn)
    sub = idx[lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
    ok = (widx >= 0)
    for c in range(2):
        vw[c * wnn + widx[ok]] = v[c * nn + sub[ok]]
    outw = O.apply_S(sw, vw)
    for c in range(2):
        a = full[c * nn + idx[cy, cx]]
        b = outw[c * wnn + widx[cy - lo[1], cx - lo[0]]]
        assert abs(a - b) <= 1e-12 * np.abs(full).max()


def test_window_helper_matches_full_apply():
    """The domain-of-dependence helper used by the full-size GPU parity tests
    reproduces the full-domain oracle S v at nodes by a free top corner and by
    a Dirichlet corner (order 4: stencil reach 4)."""
    from _helpers import window_sample
    p = inputs.cfg_layered_2d(nu=70, order=4)
    dtc = O.cfl_dt(2, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    p.omega = 2 * math.pi / (5.5 * dtc)           # N_t = 6: windows of radius 32 < the grid
    s = O.build_system(p)
    assert s.nt == 6
    v = inputs.random_vectors(p, 1, 31)[0]
    full = O.apply_S(s, v)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    for node in [(6, p.n[1] - 2), (p.n[0] - 3, 4)]:
        R = (s.nt + 2) * 4
        assert all(min(p.n[a] - 1, node[a] + R) - max(0, node[a] - R) + 1 < p.n[a] for a in range(2))
        got = window_sample(p, s.nt, v, node, reach=4)
        want = np.array([full[c * nn + idx[node[1], node[0]]] for c in range(2)])
        assert np.abs(got - want).max() <= 1e-12 * np.abs(full).max()


def test_window_helper_matches_full_apply_on_mapped_grid():
    """The same helper on a curvilinear grid: the window keeps its nodes'
    coordinates, and its metric terms differ from the full grid's only within
    4 nodes of the window's own sides, outside the sampled node's domain of
    dependence."""
    from _helpers import window_sample
    p = inputs.cfg_layered_2d(nu=70, order=4)
    L = (p.n[0] - 1) * p.h
    p.mapping = inputs.annulus_mapping(p.n, p.h, span=0.5, r0=1.5 * L, dr=L)
    dtc = O.cfl_dt_mapped(p.n, p.h, p.cfl, p.rho, p.lam, p.mu, *p.mapping)
    p.omega = 2 * math.pi / (5.5 * dtc)           # N_t = 6: windows of radius 32 < the grid
    s = O.build_system(p)
    assert s.nt == 6
    v = inputs.random_vectors(p, 1, 33)[0]
    full = O.apply_S(s, v)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    for node in [(6, p.n[1] - 2), (p.n[0] - 3, 4)]:
        R = (s.nt + 2) * 4
        assert all(min(p.n[a] - 1, node[a] + R) - max(0, node[a] - R) + 1 < p.n[a] for a in range(2))
        got = window_sample(p, s.nt, v, node, reach=4)
        want = np.array([full[c * nn + idx[node[1], node[0]]] for c in range(2)])
        assert np.abs(got - want).max() <= 1e-12 * np.abs(full).max()


def test_conjugate_residual_converges_monotonically():
    """Section 4.5 remark: conjugate residual (M inner product) reaches the
    direct solution and its residual norm never increases (unlike CG's)."""
    s = O.build_system(_case(2, 4, [0, 0, 0, 1], 1, seed=3))
    v = O.helmholtz_direct(s)
    x, info = O.cr_solve(s, tol=1e-11, maxit=500)
    assert info.converged
    assert np.linalg.norm(x - v) <= 1e-8 * np.linalg.norm(v)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-12 * h[0])


def _w_selfadjoint_indefinite(n, n_neg, seed):
    """A matrix self-adjoint in the W inner product with n_neg negative and
    n - n_neg positive eigenvalues: W^{-1/2} Q diag(l) Q^T W^{1/2}."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-2.0, -0.3, n_neg), rng.uniform(0.2, 3.0, n - n_neg)])
    mw = rng.uniform(0.5, 2.0, n)
    wh = np.sqrt(mw)
    a = ((q * lam) @ q.T) * wh[None, :] / wh[:, None]
    return a, mw, rng.standard_normal(n)


@pytest.mark.parametrize("n_neg", [0, 7, 20])
def test_minres_solves_w_selfadjoint_systems(n_neg):
    """Section 4.4 remark (MINRES for indefinite systems): on W-self-adjoint
    systems, definite or not, the oracle's MINRES reaches numpy's solution,
    terminates within n + 5 iterations (finite termination of the Krylov
    method) and its W-norm residual never increases.  Its reported residual
    is the true one."""
    n = 30
    a, mw, b = _w_selfadjoint_indefinite(n, n_neg, 7 + n_neg)
    x, info = O.minres(lambda v: a @ v, b, mw, tol=1e-12, maxit=200)
    want = np.linalg.solve(a, b)
    assert info.converged and info.iters <= n + 5
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-14)
    r = b - a @ x
    true = math.sqrt(np.dot(mw * r, r) / np.dot(mw * b, b))
    assert abs(true - info.rel_res) <= 1e-10


def test_minres_solves_indefinite_wave_holtz_system():
    """Few time steps per period (N_t = 5) near a resonance make the discrete
    filter exceed 1 on one mode (Appendix B), so M(I - S) is indefinite while
    the scheme is stable: checked here with the dense S.  MINRES still
    reaches the discrete Helmholtz solution, monotonically."""
    p = inputs.small_problem(2, [6, 5], 2, [0, 1, 0, 0], seed=3, omega=24.75)
    s = O.build_system(p, nt=5)
    S = O.form_S(s)
    mh = np.sqrt(s.Mdiag)
    a_sym = ((np.eye(S.shape[0]) - S) * mh[:, None]) / mh[None, :]
    ev = np.linalg.eigvalsh(0.5 * (a_sym + a_sym.T))
    assert ev.min() < -1e-3 and ev.max() < 1.5          # indefinite, and stable
    v = O.helmholtz_direct(s)
    x, info = O.minres_solve(s, tol=1e-11, maxit=500)
    assert info.converged
    assert np.linalg.norm(x - v) <= 1e-8 * np.linalg.norm(v)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-14)


def test_minres_on_definite_system_matches_conjugate_residual():
    """On the SPD system M(I - S) of the explicit scheme, MINRES and CR both
    minimise the M-norm residual over the same Krylov spaces, so their
    residual histories agree (to rounding) and both reach the direct solution."""
    s = O.build_system(_case(2, 4, [0, 0, 0, 1], 1, seed=3))
    v = O.helmholtz_direct(s)
    xm, im = O.minres_solve(s, tol=1e-10, maxit=500)
    xc, ic = O.cr_solve(s, tol=1e-10, maxit=500)
    assert im.converged and ic.converged
    n = min(20, len(im.history), len(ic.history))
    assert np.allclose(im.history[:n], ic.history[:n], rtol=1e-6, atol=1e-13)
    assert np.linalg.norm(xm - v) <= 1e-7 * np.linalg.norm(v)


# ---------------------------------------------------------------- implicit scheme (Section 4.4)

IMPLICIT_CASES = [(2, 2, [0, 0, 0, 1], 5), (2, 4, [1, 0, 0, 1], 12), (3, 2, [0, 0, 0, 0, 0, 1], 7)]


def _implicit(dim, order, bc, corrected=1, seed=7):
    p = _case(dim, order, bc, 1, seed=seed)
    p.implicit = 1
    p.corrected = corrected
    return p


@pytest.mark.parametrize("dim,order,bc,nt", IMPLICIT_CASES)
@pytest.mark.parametrize("corrected", [1, 0])
def test_implicit_fixed_point(dim, order, bc, nt, corrected):
    """Section 4.4: with alpha = cos(w dt)(2 + w^2 dt^2) and the modified start,
    the solution of (w^2 M - K) v = W f is an exact fixed point of Pi_h; the
    unmodified scheme (alpha = 2) converges to the Helmholtz solution at the
    shifted frequency w~ = 2 sin(w dt / 2) / (dt sqrt(cos(w dt)))."""
    s = O.build_system(_implicit(dim, order, bc, corrected), nt=nt)
    wd = s.omega * s.dt
    if corrected:
        assert abs(s.alpha - math.cos(wd) * (2 + wd * wd)) < 1e-15
        w_eff = s.omega
    else:
        assert s.alpha == 2.0
        w_eff = 2.0 * math.sin(wd / 2.0) / (s.dt * math.sqrt(math.cos(wd)))
    A = (w_eff * w_eff) * np.diag(s.Mdiag) - s.K.toarray()
    v = np.linalg.solve(A, s.Wdiag * s.f_u[0])
    assert np.linalg.norm(O.apply_Pi(s, v) - v) <= 1e-11 * np.linalg.norm(v)


@pytest.mark.parametrize("dim,order,bc,nt", IMPLICIT_CASES[:2])
def test_implicit_S_self_adjoint_and_eigenvalues(dim, order, bc, nt):
    """M (I - S) is symmetric for the implicit scheme too, and S acts on each
    eigenmode of M^{-1} K (eigenvalue k2) by sum_n w_n cos(n theta) with
    cos theta = alpha / (2 + dt^2 k2) (the mode recurrence of the scheme)."""
    s = O.build_system(_implicit(dim, order, bc), nt=nt)
    S = O.form_S(s)
    A = np.diag(s.Mdiag) @ (np.eye(S.shape[0]) - S)
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ms = np.sqrt(s.Mdiag)
    kap = np.linalg.eigvalsh(s.K.toarray() / ms[:, None] / ms[None, :])
    theta = np.arccos(s.alpha / (2.0 + s.dt ** 2 * kap))
    pred = np.sort(np.cos(np.outer(theta, np.arange(len(s.weights)))) @ s.weights)
    got = np.sort(np.linalg.eigvals(S).real)
    assert np.abs(pred - got).max() < 1e-11


def test_implicit_alpha_stability_bound():
    """Section 4.4: stability needs |alpha| < 2; alpha = cos(2 pi / k)(2 + (2 pi / k)^2)
    meets it for every k >= 5 time steps per period and fails at k = 3."""
    for k in range(5, 400):
        a = math.cos(2 * math.pi / k) * (2 + (2 * math.pi / k) ** 2)
        assert abs(a) < 2.0
    a3 = math.cos(2 * math.pi / 3) * (2 + (2 * math.pi / 3) ** 2)
    assert abs(a3) > 2.0


def test_implicit_krylov_solves():
    """CG and MINRES on the implicit scheme's system reach the direct solution."""
    s = O.build_system(_implicit(2, 2, [0, 0, 0, 1]), nt=8)
    v = O.helmholtz_direct(s)
    x, info = O.cg_solve(s, tol=1e-11, maxit=500)
    assert info.converged and np.linalg.norm(x - v) <= 1e-9 * np.linalg.norm(v)
    xm, im = O.minres_solve(s, tol=1e-11, maxit=500)
    assert im.converged and np.linalg.norm(xm - v) <= 1e-9 * np.linalg.norm(v)


def test_implicit_few_steps_is_indefinite_and_minres_solves_it():
    """The situation of the Section 4.4 remark: the implicit scheme with five
    steps per period makes M(I - S) indefinite (dense-S eigenvalues), and
    MINRES still reaches the discrete Helmholtz solution, monotonically."""
    p = inputs.small_problem(2, [6, 5], 2, [0, 1, 0, 0], seed=3, omega=7.5)
    p.implicit = 1
    s = O.build_system(p, nt=5)
    S = O.form_S(s)
    mh = np.sqrt(s.Mdiag)
    a_sym = ((np.eye(S.shape[0]) - S) * mh[:, None]) / mh[None, :]
    ev = np.linalg.eigvalsh(0.5 * (a_sym + a_sym.T))
    assert ev.min() < -1e-3 < 1e-3 < ev.max()
    v = O.helmholtz_direct(s)
    x, info = O.minres_solve(s, tol=1e-11, maxit=500)
    assert info.converged
    assert np.linalg.norm(x - v) <= 1e-8 * np.linalg.norm(v)
    assert np.all(np.diff(info.history) <= 1e-14)


# ---------------------------------------------------------------- curvilinear grids (Section 4.1)

def _grid_coords(n, h):
    return np.meshgrid(np.arange(n[0]) * h, np.arange(n[1]) * h)


def _annulus(n, h, span=math.pi / 3, r0=1.0, dr=0.5):
    """Annular sector, radius along q and angle along r (so J > 0):
    x = (r0 + dr q') cos(span r'), y = (r0 + dr q') sin(span r'), q', r' in [0, 1]."""
    Q, R = _grid_coords(n, h)
    rad = r0 + dr * Q / (h * (n[0] - 1))
    ang = span * R / (h * (n[1] - 1))
    return rad * np.cos(ang), rad * np.sin(ang)


def test_mapped_identity_is_cartesian():
    """With x = q, y = r the mapped assembly is the Cartesian order-4 operator."""
    p = inputs.small_problem(2, [10, 9], 4, [0, 1, 1, 0, 0, 0], seed=4)
    Q, R = _grid_coords(p.n, p.h)
    K1, M1, W1, _, _ = O.assemble(2, p.n, p.h, 4, p.bc, p.rho, p.lam, p.mu)
    K2, M2, W2, _, _ = O.assemble_mapped(p.n, p.h, p.bc, p.rho, p.lam, p.mu, Q, R)
    assert abs(K1 - K2).max() <= 1e-13 * abs(K1).max()
    assert np.abs(M1 - M2).max() <= 1e-14 * M1.max() and np.abs(W1 - W2).max() <= 1e-14 * W1.max()
    p.mapping = (Q, R)
    p2 = inputs.small_problem(2, [10, 9], 4, [0, 1, 1, 0, 0, 0], seed=4)
    assert O.build_system(p).nt == O.build_system(p2).nt


def test_mapped_affine_rigid_modes_and_psd():
    """On an affine (rotated, scaled, shifted) grid with every side free, the
    physical rigid motions (two translations, the rotation (-y, x)) are in the
    kernel of K to rounding, and K is symmetric positive semi-definite with
    exactly that 3-dimensional kernel."""
    p = inputs.small_problem(2, [10, 9], 4, [1, 1, 1, 1, 0, 0], seed=4)
    Q, R = _grid_coords(p.n, p.h)
    th, sc = 0.3, 1.7
    X = sc * (math.cos(th) * Q - math.sin(th) * R) + 0.2
    Y = sc * (math.sin(th) * Q + math.cos(th) * R) - 0.1
    K, M, W, _, sel = O.assemble_mapped(p.n, p.h, p.bc, p.rho, p.lam, p.mu, X, Y)
    x, y = X.reshape(-1)[sel], Y.reshape(-1)[sel]
    for u in (np.concatenate([np.ones_like(x), 0 * x]), np.concatenate([0 * x, np.ones_like(x)]),
              np.concatenate([-y, x])):
        assert np.abs(K @ u).max() <= 1e-12 * abs(K).max()
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-14 * np.abs(Kd).max()
    ev = np.linalg.eigvalsh(Kd)
    assert ev.min() >= -1e-12 * ev.max()
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 3


def test_mapped_interior_truncation_fourth_order():
    """On a curved sector grid, M^{-1} K u at interior nodes (9 or more nodes
    from every side) approximates -(1/rho) div sigma(u) of a smooth field to
    fourth order: (lambda + mu) grad div u + mu Lap u, written out by hand."""
    lam0, mu0 = 2.0, 1.0

    def exact(x, y):
        dxdiv = -0.3 * np.sin(x) * np.cos(y) - 0.4 * np.sin(2 * x) * np.cos(y)
        dydiv = -0.3 * np.cos(x) * np.sin(y) - 0.2 * np.cos(2 * x) * np.sin(y)
        lapu = -0.6 * np.sin(x) * np.cos(y)
        lapv = -1.0 * np.cos(2 * x) * np.sin(y)
        return (lam0 + mu0) * dxdiv + mu0 * lapu, (lam0 + mu0) * dydiv + mu0 * lapv

    errs = []
    for m in (33, 65):
        n = [m, m]
        h = 1.0 / (m - 1)
        X, Y = _annulus(n, h)
        ones = np.ones((m, m))
        K, M, W, rho_u, sel = O.assemble_mapped(n, h, [1, 1, 1, 1], ones, lam0 * ones, mu0 * ones, X, Y)
        x, y = X.reshape(-1)[sel], Y.reshape(-1)[sel]
        u = np.concatenate([0.3 * np.sin(x) * np.cos(y), 0.2 * np.cos(2 * x) * np.sin(y)])
        got = -(K @ u) / M
        ex, ey = exact(x, y)
        ii, jj = np.meshgrid(np.arange(m), np.arange(m))
        inner = ((ii >= 9) & (ii <= m - 10) & (jj >= 9) & (jj <= m - 10)).reshape(-1)[sel]
        nn = len(sel)
        err = max(np.abs(got[:nn] - ex)[inner].max(), np.abs(got[nn:] - ey)[inner].max())
        errs.append(err)
    rate = math.log2(errs[0] / errs[1])
    assert rate > 3.6, (errs, rate)


def test_mapped_cfl_stable_and_fixed_point():
    """On the sector grid with cfl = 0.5 the leapfrog bound c dt^2 rho(M^{-1} K) < 4
    holds with margin, and the Helmholtz solution is a fixed point of Pi."""
    p = inputs.small_problem(2, [12, 12], 4, [0, 1, 0, 0, 0, 0], seed=9)
    n = p.n
    h = 1.0 / (n[0] - 1)
    p.h = h
    p.mapping = _annulus(n, h)
    s = O.build_system(p)
    ms = np.sqrt(s.Mdiag)
    top = np.linalg.eigvalsh(s.K.toarray() / ms[:, None] / ms[None, :]).max()
    assert O.mapped_metrics(n, h, *p.mapping)[0].min() > 0
    assert s.kt * top < 2.0
    v = O.helmholtz_direct(s)
    assert np.linalg.norm(O.apply_Pi(s, v) - v) <= 1e-11 * np.linalg.norm(v)


@pytest.mark.parametrize("mapper,bc", [("annulus", [0, 1, 1, 0, 0, 0]), ("wavy", [1, 1, 0, 1, 0, 0])])
def test_mapped_S_is_M_selfadjoint_with_filter_spectrum(mapper, bc):
    """On mapped grids (Section 4.1, curvilinear form) the WaveHoltz operator
    keeps the structure of Sections 3 and 4.5: M(I - S) is symmetric, the
    eigenvalues of A lie in (0, 3/2), and S acts on each eigenmode of
    M^{-1}K by sum_n w_n cos(n theta), cos theta = 1 - c dt^2 k2 / 2."""
    p = inputs.small_problem(2, [9, 8], 4, bc, seed=8)
    p.mapping = (inputs.annulus_mapping if mapper == "annulus" else inputs.wavy_mapping)(p.n, p.h)
    s = O.build_system(p)
    S = O.form_S(s)
    MA = s.Mdiag[:, None] * (np.eye(S.shape[0]) - S)
    assert np.abs(MA - MA.T).max() <= 1e-13 * np.abs(MA).max()
    Ms = np.sqrt(s.Mdiag)
    ev = np.linalg.eigvalsh(0.5 * (MA + MA.T) / Ms[:, None] / Ms[None, :])
    g = _golden_kv("section3_filter.txt")
    assert ev.min() > g["A_eig_lower"] and ev.max() < g["A_eig_upper"]
    kap = np.linalg.eigvalsh(s.K.toarray() / Ms[:, None] / Ms[None, :])
    theta = np.arccos(1.0 - s.kt * kap / 2.0)
    pred = np.sort(np.cos(np.outer(theta, np.arange(len(s.weights)))) @ s.weights)
    got = np.sort(np.linalg.eigvals(S).real)
    assert np.abs(pred - got).max() < 1e-11


@pytest.mark.parametrize("variant", ["periods2", "implicit", "uncorrected_implicit"])
def test_mapped_fixed_point_with_other_forms(variant):
    """The mapped operator composes with the other forms of the method: with
    the K = 2 filter (Section 3, many-periods filter) and with the implicit
    time-corrected scheme (Section 4.4) the Helmholtz solution on the sector
    grid is a fixed point of Pi (with the paper's shifted frequency for the
    unmodified implicit scheme)."""
    p = inputs.small_problem(2, [10, 9], 4, [0, 1, 1, 0, 0, 0], seed=12)
    p.mapping = inputs.annulus_mapping(p.n, p.h)
    nt = 0
    if variant == "periods2":
        p.periods = 2
    else:
        p.implicit = 1
        nt = 8
        if variant == "uncorrected_implicit":
            p.corrected = 0
    s = O.build_system(p, nt=nt) if nt else O.build_system(p)
    v = O.helmholtz_direct(s)
    assert np.linalg.norm(O.apply_Pi(s, v) - v) <= 1e-11 * np.linalg.norm(v)


def test_mapped_mms_rate_with_traction_free_curved_side():
    """Manufactured solution on an annular sector whose outer arc is traction
    free (Section 4.1, curvilinear form; the free side is the natural
    boundary condition of the mapped energy).  In polar coordinates
    u = (r - R0)(r - R1)^2 [sin(pi th / Th) e_r + sin(2 pi th / Th) e_th / 2]
    vanishes on the inner arc and both radial sides, and its stresses vanish
    on the outer arc r = R1 (the double zero removes both u and its radial
    derivative there), so it solves rho w^2 u + div T(u) = f with exactly the
    discrete problem's boundary conditions.  The discrete Helmholtz solution
    converges to it at third order or better (fourth-order interior, SBP
    closure and metric terms of second order at the sides)."""
    sy = pytest.importorskip("sympy")
    X, Y = sy.symbols("x y")
    R0, R1, Th, lam0, mu0, rho0, omega = 1.0, 1.5, math.pi / 3, 2.0, 1.0, 1.0, 1.3
    r = sy.sqrt(X ** 2 + Y ** 2)
    th = sy.atan2(Y, X)
    g = (r - R0) * (r - R1) ** 2
    ur, ut = g * sy.sin(sy.pi * th / Th), g * sy.sin(2 * sy.pi * th / Th) / 2
    uex = ur * sy.cos(th) - ut * sy.sin(th)
    vex = ur * sy.sin(th) + ut * sy.cos(th)
    ux, uy, vx, vy = sy.diff(uex, X), sy.diff(uex, Y), sy.diff(vex, X), sy.diff(vex, Y)
    sxx = lam0 * (ux + vy) + 2 * mu0 * ux
    syy = lam0 * (ux + vy) + 2 * mu0 * vy
    sxy = mu0 * (uy + vx)
    # the traction on the outer arc vanishes (checked symbolically at a point)
    nx, ny = sy.cos(th), sy.sin(th)
    pt = {X: R1 * math.cos(0.4), Y: R1 * math.sin(0.4)}
    assert abs(float((sxx * nx + sxy * ny).subs(pt))) < 1e-12
    assert abs(float((sxy * nx + syy * ny).subs(pt))) < 1e-12
    fx = rho0 * omega ** 2 * uex + sy.diff(sxx, X) + sy.diff(sxy, Y)
    fy = rho0 * omega ** 2 * vex + sy.diff(sxy, X) + sy.diff(syy, Y)
    fns = [sy.lambdify((X, Y), e, "numpy") for e in (fx, fy, uex, vex)]
    errs = []
    ms = (17, 33, 65)
    for m in ms:
        n = [m, m]
        h = 1.0 / (m - 1)
        Xg, Yg = _annulus(n, h, span=Th, r0=R0, dr=R1 - R0)
        ones = np.ones((m, m))
        ev = [np.asarray(f(Xg, Yg), dtype=float) for f in fns]
        prob = inputs.Problem("mms_sector", 2, n, h, 4, [0, 1, 0, 0, 0, 0], omega, rho0 * ones, lam0 * ones,
                              mu0 * ones, np.stack([np.stack([ev[0], ev[1]])]))
        prob.mapping = (Xg, Yg)
        s = O.build_system(prob)
        vnum = O.helmholtz_direct(s)
        ex = np.concatenate([ev[2].reshape(-1)[s.sel], ev[3].reshape(-1)[s.sel]])
        errs.append(np.abs(vnum - ex).max())
    rates = [math.log(errs[i] / errs[i + 1]) / math.log((ms[i + 1] - 1) / (ms[i] - 1)) for i in range(2)]
    assert rates[-1] > 2.7, (errs, rates)
