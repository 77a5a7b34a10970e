"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 GPU results must match the oracle within 1e-10 relative; FP32-stencil
results within tests/_helpers.tol32(N).  Inputs are the seeded generators of
paper_2205_12344_gb300.inputs, identical on both sides.
"""
import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import TOL64, oracle_all_rhs, rel_err, to_np, tol32, window_sample

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _wh(prob, precision="fp64", nt=0):
    from paper_2205_12344_gb300.api import WaveHoltz
    return WaveHoltz(prob, precision=precision, nt=nt)


# (dim, interior nodes per axis, order, bc, nrhs): odd sizes, every side type,
# tiles with ragged tails (32 x 8 and 32 x 4 x 2 tiles), several rhs
CASES = [
    (2, [5, 7], 2, [0, 0, 0, 0], 1),
    (2, [37, 11], 2, [0, 0, 0, 1], 2),
    (2, [9, 40], 2, [1, 0, 1, 0], 1),
    (2, [33, 17], 2, [1, 1, 1, 1], 1),
    (2, [2, 2], 2, [0, 0, 0, 0], 1),
    (2, [8, 9], 4, [0, 0, 0, 0], 1),
    (2, [41, 13], 4, [0, 0, 0, 1], 3),
    (2, [12, 35], 4, [1, 1, 0, 1], 1),
    (2, [6, 6], 4, [1, 1, 1, 1], 1),
    (3, [5, 6, 7], 2, [0, 0, 0, 0, 0, 0], 1),
    (3, [35, 5, 4], 2, [0, 0, 1, 0, 0, 1], 2),
    (3, [7, 6, 8], 4, [0, 0, 0, 0, 0, 1], 1),
    (3, [9, 6, 6], 4, [1, 0, 0, 1, 1, 0], 1),
]


def _ids(c):
    return "d%d_%s_o%d_bc%s_r%d" % (c[0], "x".join(map(str, c[1])), c[2], "".join(map(str, c[3][:2 * c[0]])), c[4])


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_setup_and_operator_match_oracle(case):
    dim, nu, order, bc, nrhs = case
    p = inputs.small_problem(dim, nu, order, bc, seed=11, nrhs=nrhs)
    s = O.build_system(p)
    with _wh(p) as wh:
        assert wh.info.nt == s.nt
        assert abs(wh.info.kt - s.kt) <= 1e-15 * s.kt
        assert abs(wh.info.omega_tilde - s.omega_tilde) <= 1e-14 * s.omega_tilde
        assert wh.info.n_unknowns == s.K.shape[0]
        u = inputs.random_vectors(p, 1, 5)[0]
        got = to_np(wh.apply_minvK(u))
        want = oracle_all_rhs(s, lambda ss, x, r: O.minv_K(ss, x), u)
        assert rel_err(got, want) < 1e-12


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_apply_S_and_Pi0_fp64_match_oracle(case):
    dim, nu, order, bc, nrhs = case
    p = inputs.small_problem(dim, nu, order, bc, seed=12, nrhs=nrhs)
    s = O.build_system(p)
    with _wh(p) as wh:
        v = inputs.random_vectors(p, 1, 6)[0]
        got = to_np(wh.apply_S(v))
        want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
        assert rel_err(got, want) < TOL64
        b = to_np(wh.apply_Pi0())
        bw = np.concatenate([O.apply_Pi0(s, r) for r in range(nrhs)])
        assert rel_err(b, bw) < TOL64
        # aliasing input and output is allowed
        vt = wh._vec(v)
        from paper_2205_12344_gb300 import _lib as L
        L.ewh_apply_S(wh.ctx, vt, vt)
        assert rel_err(to_np(vt), want) < TOL64


@pytest.mark.parametrize("case", [c for c in CASES if c[1] != [2, 2]], ids=[_ids(c) for c in CASES if c[1] != [2, 2]])
def test_apply_S_fp32_within_stated_tolerance(case):
    dim, nu, order, bc, nrhs = case
    p = inputs.small_problem(dim, nu, order, bc, seed=13, nrhs=nrhs)
    s = O.build_system(p)
    with _wh(p, "fp32") as wh:
        v = inputs.random_vectors(p, 1, 7)[0]
        got = to_np(wh.apply_S(v))
        want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
        assert rel_err(got, want) < tol32(s.nt), rel_err(got, want)
        got64 = to_np(wh.apply_S(v, fp64=True))
        assert rel_err(got64, want) < TOL64


@pytest.mark.parametrize("periods", [1, 2])
def test_periods_and_uncorrected_match_oracle(periods):
    p = inputs.small_problem(2, [20, 13], 4, [0, 0, 0, 1], seed=3)
    p.periods = periods
    for corrected in (1, 0):
        p.corrected = corrected
        s = O.build_system(p)
        with _wh(p) as wh:
            v = inputs.random_vectors(p, 1, 8)[0]
            assert rel_err(to_np(wh.apply_S(v)), O.apply_S(s, v)) < TOL64


def test_explicit_nt_matches_oracle():
    p = inputs.small_problem(2, [10, 11], 2, [0, 0, 0, 1], seed=4)
    s = O.build_system(p, nt=7)
    with _wh(p, nt=7) as wh:
        assert wh.info.nt == 7
        v = inputs.random_vectors(p, 1, 9)[0]
        assert rel_err(to_np(wh.apply_S(v)), O.apply_S(s, v)) < TOL64


def test_mdot_matches_oracle():
    p = inputs.small_problem(2, [30, 21], 4, [0, 0, 0, 1], seed=5, nrhs=2)
    s = O.build_system(p)
    x, y = inputs.random_vectors(p, 2, 10)
    n = s.K.shape[0]
    with _wh(p) as wh:
        got = wh.mdot(x, y)
        for r in range(2):
            want = O.mdot(s, x[r * n:(r + 1) * n], y[r * n:(r + 1) * n])
            assert abs(got[r] - want) <= 1e-12 * abs(want) + 1e-14


# ---------------------------------------------------------------- solves

def test_solve_fp64_matches_oracle_cg_homogeneous():
    """The homogeneous 2D configuration at reduced size (32x32, w = 10): same
    iterates as the oracle CG and the direct Helmholtz solution."""
    p = inputs.cfg_homogeneous_2d(nu=32, omega=10.0)
    s = O.build_system(p)
    xo, info_o = O.cg_solve(s, tol=1e-8)
    v_direct = O.helmholtz_direct(s)
    with _wh(p) as wh:
        x, info = wh.solve(tol=1e-8)
        hist = wh.residual_history()
    assert info.status == 0
    assert abs(info.iters - info_o.iters) <= 1
    n = min(20, len(hist), len(info_o.history))
    assert np.allclose(hist[:n], info_o.history[:n], rtol=1e-7, atol=0)
    assert rel_err(to_np(x), xo) < 1e-7
    assert info.rel_res <= 1e-8
    assert np.linalg.norm(to_np(x) - v_direct) / np.linalg.norm(v_direct) < 1e-5


@pytest.mark.parametrize("order,bc", [(2, [0, 0, 0, 1]), (4, [0, 0, 0, 1]), (4, [1, 0, 0, 0])])
def test_solve_fp64_matches_direct(order, bc):
    p = inputs.small_problem(2, [24, 19], order, bc, seed=2, nrhs=2)
    s = O.build_system(p)
    with _wh(p) as wh:
        x, info = wh.solve(tol=1e-11, maxit=2000)
    n = s.K.shape[0]
    for r in range(2):
        v = O.helmholtz_direct(s, r)
        assert np.linalg.norm(to_np(x)[r * n:(r + 1) * n] - v) <= 1e-8 * np.linalg.norm(v)


@pytest.mark.parametrize("order", [2, 4])
def test_solve_fp32_stencil_reaches_fp64_residual(order):
    p = inputs.cfg_homogeneous_2d(nu=40, omega=12.0, order=order)
    with _wh(p) as wh64:
        x64, i64 = wh64.solve(tol=1e-10)
    with _wh(p, "fp32") as wh:
        x, info = wh.solve(tol=1e-8)
        # the reported residual is the FP64 one: recompute it independently
        vb = to_np(wh64_b(p))
        r = vb - (to_np(x) - to_np(wh.apply_S(x, fp64=True)))
        s = O.build_system(p)
        rel = np.sqrt(O.mdot(s, r, r) / O.mdot(s, vb, vb))
    assert info.status == 0
    assert info.rel_res <= 1e-8
    assert rel <= 1.01e-8
    assert rel_err(to_np(x), to_np(x64)) < 1e-6


def wh64_b(p):
    with _wh(p) as wh:
        return wh.apply_Pi0()


def test_solve_with_initial_guess():
    p = inputs.cfg_homogeneous_2d(nu=24, omega=8.0)
    s = O.build_system(p)
    v = O.helmholtz_direct(s)
    with _wh(p) as wh:
        x, info = wh.solve(tol=1e-9, x0=v * (1 + 1e-3))
        x0, info0 = wh.solve(tol=1e-9)
    assert info.iters < info0.iters
    assert rel_err(to_np(x), v) < 1e-6


def test_solve_without_forcing_is_rejected():
    from paper_2205_12344_gb300.api import WaveHoltz
    from paper_2205_12344_gb300 import _lib as L
    p = inputs.small_problem(2, [8, 8], 2, [0, 0, 0, 0], seed=1)
    wh = WaveHoltz(p, forcing=False)
    with pytest.raises(L.EwhError) as e:
        wh.solve()
    assert e.value.status == L.EWH_EINVAL
    wh.close()


# ---------------------------------------------------------------- full size

def test_layered_1024_fp32_sampled_parity_and_symmetry():
    """The benchmark workload (2D layered 1024^2, order 4, free top, FP32
    stencil, launch configuration of bench.py): S v at a node by the free top
    near a Dirichlet side from the oracle on its domain of dependence, and the
    symmetry (x, S y)_M = (y, S x)_M of eq. (amat_sym)."""
    import math
    p = inputs.cfg_layered_2d(nu=1024, order=4)
    from paper_2205_12344_gb300.api import WaveHoltz
    with WaveHoltz(p, precision="fp32") as wh:
        nt = wh.info.nt
        v = inputs.random_vectors(p, 1, 21)[0]
        got = to_np(wh.apply_S(v))
        x, y = inputs.random_vectors(p, 2, 22)
        Sx = wh.apply_S(x)
        Sy = wh.apply_S(y)
        a = wh.mdot(x, Sy)[0]
        b = wh.mdot(y, Sx)[0]
        assert abs(a - b) <= 1e-5 * math.sqrt(wh.mdot(x, x)[0] * wh.mdot(y, y)[0])
    dtc = O.cfl_dt(2, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    assert nt == max(5, int(math.ceil(2 * math.pi / p.omega / dtc)))
    node = (6, p.n[1] - 2)
    want = window_sample(p, nt, v, node, reach=4)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    gv = np.array([got[c * nn + idx[node[1], node[0]]] for c in range(2)])
    scale = np.abs(got).max()
    assert np.abs(gv - want).max() <= tol32(nt) * scale, (gv, want)


def test_layered_1024_fp64_sampled_parity():
    """Same workload in FP64: the sampled entry within 1e-10 of the oracle."""
    p = inputs.cfg_layered_2d(nu=1024, order=4)
    from paper_2205_12344_gb300.api import WaveHoltz
    with WaveHoltz(p, precision="fp64") as wh:
        nt = wh.info.nt
        v = inputs.random_vectors(p, 1, 23)[0]
        got = to_np(wh.apply_S(v))
    node = (p.n[0] - 3, 4)      # by the Dirichlet bottom-right corner
    want = window_sample(p, nt, v, node, reach=4)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    gv = np.array([got[c * nn + idx[node[1], node[0]]] for c in range(2)])
    assert np.abs(gv - want).max() <= TOL64 * np.abs(got).max(), (gv, want)


@pytest.mark.parametrize("bc,nrhs", [([0, 1, 1, 0, 0, 1], 2), ([1, 1, 1, 1, 1, 1], 1)])
def test_order4_3d_interior_blocks_match_oracle(bc, nrhs):
    """A 3D order-4 grid large enough (72 x 24 x 14 nodes) that some 32 x 8
    blocks and planes lie in rows, columns and planes 4 .. n - 5, so the
    step kernels' central-difference fast path runs beside the closure path:
    S, Pi 0 (FP64) and S (FP32) against the oracle."""
    p = inputs.small_problem(3, [70, 22, 12], 4, bc, seed=23, nrhs=nrhs)
    assert p.n[0] >= 68 and p.n[1] >= 20 and p.n[2] >= 9   # an interior block exists
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 24)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(p.nrhs)])
    with _wh(p) as wh:
        assert rel_err(to_np(wh.apply_S(v)), want) < TOL64
        assert rel_err(to_np(wh.apply_Pi0()), want0) < TOL64
        u = inputs.random_vectors(p, 1, 25)[0]
        kw = oracle_all_rhs(s, lambda ss, x, r: O.minv_K(ss, x), u)
        assert rel_err(to_np(wh.apply_minvK(u)), kw) < 1e-12
    with _wh(p, "fp32") as wh:
        assert rel_err(to_np(wh.apply_S(v)), want) < tol32(s.nt)


@pytest.mark.parametrize("variant", ["split", "fused"])
@pytest.mark.parametrize("shape", [[45, 19], [70, 131]])
def test_order4_2d_kernel_variants_match_oracle(variant, shape, monkeypatch):
    """Every 2D order-4 step kernel (stress + divergence launches with their
    interior shared-memory tiles, and the fused tile launch) reproduces the
    oracle S apply, FP64 and FP32, on grids with interior and boundary blocks
    and ragged tails."""
    monkeypatch.setenv("EWH_STEP2D_O4", variant)
    p = inputs.small_problem(2, shape, 4, [1, 0, 0, 1], seed=17, nrhs=2)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 18)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    with _wh(p) as wh:
        assert rel_err(to_np(wh.apply_S(v)), want) < TOL64
        kinds = wh.kernel_launches()
    with _wh(p, "fp32") as wh:
        assert rel_err(to_np(wh.apply_S(v)), want) < tol32(s.nt)
    assert kinds > 0


def test_conjugate_residual_matches_oracle():
    """ewh_solve_cr (FP64) follows the oracle's conjugate residual iterates and
    reaches the direct solution; the FP32-stencil variant meets the FP64
    residual tolerance."""
    p = inputs.cfg_homogeneous_2d(nu=32, omega=10.0)
    s = O.build_system(p)
    xo, io = O.cr_solve(s, tol=1e-9)
    v = O.helmholtz_direct(s)
    with _wh(p) as wh:
        x, info = wh.solve_cr(tol=1e-9)
        hist = wh.residual_history()
    assert info.status == 0 and abs(info.iters - io.iters) <= 1
    n = min(15, len(hist), len(io.history))
    assert np.allclose(hist[:n], io.history[:n], rtol=1e-7, atol=0)
    assert rel_err(to_np(x), xo) < 1e-6
    assert np.linalg.norm(to_np(x) - v) <= 1e-6 * np.linalg.norm(v)
    with _wh(p, "fp32") as wh:
        x32, i32 = wh.solve_cr(tol=1e-8)
    assert i32.status == 0 and i32.rel_res <= 1e-8


def test_minres_matches_oracle():
    """ewh_solve_minres (FP64) follows the oracle's MINRES residual history and
    reaches the direct solution; the FP32-stencil variant meets the FP64
    residual tolerance (Section 4.4 remark)."""
    p = inputs.cfg_homogeneous_2d(nu=32, omega=10.0)
    s = O.build_system(p)
    xo, io = O.minres_solve(s, tol=1e-9)
    v = O.helmholtz_direct(s)
    with _wh(p) as wh:
        x, info = wh.solve_minres(tol=1e-9)
        hist = wh.residual_history()
    assert info.status == 0 and abs(info.iters - io.iters) <= 1
    n = min(15, len(hist), len(io.history))
    assert np.allclose(hist[:n], io.history[:n], rtol=1e-7, atol=0)
    assert np.all(np.diff(hist[:n]) <= 1e-12)
    assert np.linalg.norm(to_np(x) - v) <= 1e-6 * np.linalg.norm(v)
    with _wh(p, "fp32") as wh:
        x32, i32 = wh.solve_minres(tol=1e-8)
    assert i32.status == 0 and i32.rel_res <= 1e-8
    assert rel_err(to_np(x32), v) < 1e-5


def test_minres_solves_indefinite_system():
    """N_t = 5 near a resonance: M(I - S) is indefinite (the oracle test pins
    that with the dense S) yet the stable scheme's fixed point is the discrete
    Helmholtz solution.  GPU MINRES reaches it with a non-increasing residual."""
    p = inputs.small_problem(2, [6, 5], 2, [0, 1, 0, 0], seed=3, omega=24.75)
    s = O.build_system(p, nt=5)
    v = O.helmholtz_direct(s)
    with _wh(p, nt=5) as wh:
        assert wh.info.nt == 5
        x, info = wh.solve_minres(tol=1e-11, maxit=500)
        hist = wh.residual_history()
    assert info.status == 0 and info.rel_res <= 1e-11
    assert np.all(np.diff(hist) <= 1e-12)
    assert np.linalg.norm(to_np(x) - v) <= 1e-8 * np.linalg.norm(v)


def test_cg_continues_with_minres_on_indefinite_system():
    """CG on the same indefinite system meets (p, A p)_M <= 0 (at its 26th
    iteration in the oracle's arithmetic); ewh_solve continues from that
    iterate with MINRES (Section 4.4 remark) and reaches the discrete
    Helmholtz solution, counting the MINRES iterations apart."""
    p = inputs.small_problem(2, [6, 5], 2, [0, 1, 0, 0], seed=3, omega=24.75)
    s = O.build_system(p, nt=5)
    v = O.helmholtz_direct(s)
    with _wh(p, nt=5) as wh:
        x, info = wh.solve(tol=1e-11, maxit=500)
    assert info.status == 0 and info.rel_res <= 1e-11
    assert 0 < info.minres_iters < info.iters
    assert np.linalg.norm(to_np(x) - v) <= 1e-8 * np.linalg.norm(v)
