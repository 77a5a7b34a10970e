"""The on-chip resident wave solve (2D, order-4 SBP, FP32 stencil: every
leapfrog level of S in one cooperative launch per group of right-hand sides,
the state in shared memory and registers, halos exchanged through global
memory at one grid barrier per level) against the oracle, for one and
several right-hand sides and for batch members.

EWH_STEP2D_O4=r<k> selects CTA shape k (1024 x 7, 768 x 9, 512 x 14 threads
x nodes per thread) when the grid fits it; each test checks that the chosen
variant really is the resident one.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import oracle_all_rhs, rel_err, to_np, tol32, window_sample

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VARIANT_RESIDENT = 5
D, F = inputs.DIRICHLET, inputs.FREE


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _fp32(prob, nt=0):
    from paper_2205_12344_gb300.api import WaveHoltz
    return WaveHoltz(prob, precision="fp32", nt=nt)


def _variant(wh):
    from paper_2205_12344_gb300 import _lib as L
    return L.ewh_get_info(wh.ctx).kernel_variant[1]


# grids with several CTAs per axis, ragged last blocks and every side type
SHAPES = [([45, 19], [D, D, D, F]), ([70, 131], [F, D, D, F]), ([24, 24], [F, F, F, F]),
          ([129, 37], [D, F, F, D]), ([8, 200], [D, D, F, F])]


@pytest.mark.parametrize("shape", [0, 2])
@pytest.mark.parametrize("grid,bc", SHAPES, ids=lambda x: "x".join(map(str, x)) if isinstance(x[0], int) else "")
def test_resident_S_and_Pi0_match_oracle(grid, bc, shape, monkeypatch):
    """S v and Pi 0 (forced) of the resident launch against the oracle (eq. qoper)."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r%d" % shape)
    p = inputs.small_problem(2, grid, 4, bc + [0, 0], seed=31 + shape)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 32)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = O.apply_Pi0(s)
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
        assert _variant(wh) == VARIANT_RESIDENT + shape
        assert wh.kernel_launches() > 0
    assert rel_err(got, want) < tol32(s.nt)
    assert rel_err(got0, want0) < tol32(s.nt)


@pytest.mark.parametrize("periods", [1, 3])
def test_resident_periods_and_uncorrected(periods, monkeypatch):
    """Several periods (eq. many_periods_filter) and the uncorrected scheme."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r0")
    p = inputs.small_problem(2, [33, 27], 4, [D, F, D, F, 0, 0], seed=40)
    p.periods = periods
    p.corrected = 0 if periods == 3 else 1
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 41)[0]
    want = O.apply_S(s, v)
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        assert _variant(wh) == VARIANT_RESIDENT
    assert rel_err(got, want) < tol32(s.nt * periods)


def test_resident_solve_matches_oracle_cg(monkeypatch):
    """The mixed-precision CG solve on top of the resident S reaches the
    oracle's solution of M(I - S) v = M Pi 0 (eq. amat_sym)."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r0")
    p = inputs.small_problem(2, [40, 34], 4, [D, D, D, F, 0, 0], seed=42)
    s = O.build_system(p)
    xo, io = O.cg_solve(s, tol=1e-9)
    with _fp32(p) as wh:
        x, info = wh.solve(tol=1e-8)
        assert _variant(wh) == VARIANT_RESIDENT
    assert info.status == 0 and info.rel_res <= 1e-8
    # the oracle's own FP64 residual of the returned x
    x = to_np(x)
    b = O.apply_Pi0(s)
    r = b - (x - O.apply_S(s, x))
    assert math.sqrt(O.mdot(s, r, r) / O.mdot(s, b, b)) <= 1.01e-8
    # both solutions within the conditioning of the 1e-8 / 1e-9 stopping rules:
    # ||x - xo||_M <= kappa(A) (1e-8 + 1e-9) ||xo||_M, kappa from S's spectrum
    # (1 - beta over the eigenvalues of M^{-1} K; about 1.3e5 here)
    d = x - xo
    assert math.sqrt(O.mdot(s, d, d) / O.mdot(s, xo, xo)) <= _kappa(s, p) * 1.1e-8


def _kappa(s, p):
    """Condition number of A = I - S in the M inner product from the dense
    spectrum of M^{-1} K: eig(S) = beta(theta_j), cos theta_j = 1 - k_t lambda_j / 2."""
    ms = np.sqrt(s.Mdiag)
    lam = np.linalg.eigvalsh(s.K.toarray() / ms[:, None] / ms[None, :])
    w = O.filter_weights(s.nt, p.periods)
    th = np.arccos(np.clip(1 - s.kt * lam / 2, -1, 1))
    a = 1 - np.cos(np.outer(th, np.arange(len(w)))) @ w
    return a.max() / a.min()


def test_resident_matches_split_kernels(monkeypatch):
    """Resident and per-level split launches give the same S v to FP32
    rounding on a grid spanning many CTAs."""
    p = inputs.small_problem(2, [300, 210], 4, [F, D, D, F, 0, 0], seed=43)
    v = inputs.random_vectors(p, 1, 44)[0]
    monkeypatch.setenv("EWH_STEP2D_O4", "split")
    with _fp32(p) as wh:
        a = to_np(wh.apply_S(v))
        assert _variant(wh) < VARIANT_RESIDENT
        nt = wh.info.nt
    monkeypatch.setenv("EWH_STEP2D_O4", "r2")
    with _fp32(p) as wh:
        b = to_np(wh.apply_S(v))
        assert _variant(wh) == VARIANT_RESIDENT + 2
    assert rel_err(b, a) < 2 * tol32(nt)


@pytest.mark.parametrize("shape", [0, 2])
@pytest.mark.parametrize("grid,bc,nrhs", [([45, 19], [D, D, D, F], 3), ([70, 131], [F, D, D, F], 2)],
                         ids=["45x19r3", "70x131r2"])
def test_resident_several_rhs_match_oracle(grid, bc, nrhs, shape, monkeypatch):
    """A multi-rhs context on chip: one cooperative launch carries the blocks
    of every right-hand side; S v and Pi 0 (forced, eq. qoper) of each rhs
    against the oracle."""
    from paper_2205_12344_gb300 import _lib as L
    monkeypatch.setenv("EWH_STEP2D_O4", "r%d" % shape)
    p = inputs.small_problem(2, grid, 4, bc + [0, 0], seed=45 + shape, nrhs=nrhs)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 46)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(nrhs)])
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
        assert _variant(wh) == VARIANT_RESIDENT + shape
        plan = list(L.ewh_get_info(wh.ctx).resident)
    assert plan[8] == nrhs and plan[9] == 1  # every rhs in one launch
    assert rel_err(got, want) < tol32(s.nt)
    assert rel_err(got0, want0) < tol32(s.nt)


@pytest.fixture(scope="module")
def member256_nt6():
    """A batch member's size: layered 256^2 with 22 shots, w raised so that
    N_t = 6; one random input vector per shot."""
    shots = [0.1 + 0.11 * k for k in range(22)]
    p = inputs.cfg_layered_2d(nu=256, order=4, nrhs=22, shot_x=shots)
    dtc = O.cfl_dt(2, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    p.omega = 2 * math.pi / (5.5 * dtc)
    v = inputs.random_vectors(p, 1, 53)[0]
    return p, v


def test_resident_rhs_groups_match_split_and_oracle(member256_nt6, monkeypatch):
    """22 right-hand sides of 256^2 do not fit one co-resident launch: they
    run as groups of launches, one after another.  Every node of every rhs
    against the oracle-checked split kernels, and nodes of the first and last
    rhs (by the free top, a Dirichlet side, a CTA seam) against the oracle on
    their domains of dependence."""
    from paper_2205_12344_gb300 import _lib as L
    p, v = member256_nt6
    monkeypatch.setenv("EWH_STEP2D_O4", "split")
    with _fp32(p) as wh:
        a = to_np(wh.apply_S(v))
    monkeypatch.setenv("EWH_STEP2D_O4", "r1")
    with _fp32(p) as wh:
        b = to_np(wh.apply_S(v))
        info = L.ewh_get_info(wh.ctx)
        assert info.kernel_variant[1] == VARIANT_RESIDENT + 1 and info.nt == 6
        plan = list(info.resident)
    rg, groups = plan[8], plan[9]
    assert groups >= 2 and rg * groups >= p.nrhs and rg * (groups - 1) < p.nrhs, plan
    assert rel_err(b, a) < 2 * tol32(6)
    nn = p.n_nodes()
    n1 = 2 * nn
    idx = inputs.unknown_index(p)
    by = plan[5]
    scale = np.abs(b).max()
    for r in (0, p.nrhs - 1):
        pr = inputs.cfg_layered_2d(nu=256, order=4, nrhs=1, shot_x=[0.1 + 0.11 * r])
        pr.omega = p.omega
        vr = v[r * n1:(r + 1) * n1]
        for node in [(128, p.n[1] - 2), (1, 100), (200, by - 1), (200, by)]:
            want = window_sample(pr, 6, vr, node, reach=4)
            g = np.array([b[r * n1 + c * nn + idx[node[1], node[0]]] for c in range(2)])
            assert np.abs(g - want).max() <= tol32(6) * scale, (r, node, g, want)


def test_resident_batch_members_run_serially_and_match_single(monkeypatch):
    """Batch members on chip: the batch graph runs their cooperative launches
    one after another; every member's S v equals the same problem alone
    (bitwise) and the oracle, and the batched FP32 solve reaches an FP64
    residual the oracle confirms."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r0")
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    probs = [inputs.small_problem(2, [40, 34], 4, [D, D, D, F, 0, 0], seed=42, nrhs=2, omega=6.0),
             inputs.small_problem(2, [30, 30], 4, [D, D, D, F, 0, 0], seed=47, omega=5.0)]
    vs = [inputs.random_vectors(p, 1, 48 + k)[0] for k, p in enumerate(probs)]
    with WaveHoltzBatch(probs, "fp32") as wb:
        outs = [to_np(o) for o in wb.apply_S(vs)]
        for k in range(len(probs)):
            assert L.ewh_get_info(L.ewh_batch_member(wb.b, k)).kernel_variant[1] == VARIANT_RESIDENT
        xs, infos = wb.solve(tol=1e-7, maxit=4000)
    for p, v, o, x, inf in zip(probs, vs, outs, xs, infos):
        with _fp32(p) as wh:
            single = to_np(wh.apply_S(v))
            assert _variant(wh) == VARIANT_RESIDENT
        assert np.array_equal(o, single)
        s = O.build_system(p)
        assert rel_err(o, oracle_all_rhs(s, lambda ss, xx, r: O.apply_S(ss, xx, r), v)) < tol32(s.nt)
        assert inf.status == 0 and inf.rel_res <= 1e-7
        n = s.K.shape[0]
        x = to_np(x)
        for r in range(p.nrhs):
            b = O.apply_Pi0(s, r)
            xr = x[r * n:(r + 1) * n]
            res = b - (xr - O.apply_S(s, xr, r))
            assert math.sqrt(O.mdot(s, res, res) / O.mdot(s, b, b)) <= 1.01e-7


@pytest.mark.parametrize("shape", [0, 2])
def test_resident_layered_1024_sampled_parity(shape, monkeypatch):
    """The benchmark workload (2D layered 1024^2, order 4, free top) through the
    resident launch: S v at a node by the free top from the oracle on its
    domain of dependence (which spans many CTA blocks), and the M-symmetry of
    eq. (amat_sym)."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r%d" % shape)
    p = inputs.cfg_layered_2d(nu=1024, order=4)
    with _fp32(p) as wh:
        nt = wh.info.nt
        v = inputs.random_vectors(p, 1, 51)[0]
        got = to_np(wh.apply_S(v))
        assert _variant(wh) == VARIANT_RESIDENT + shape
        x, y = inputs.random_vectors(p, 2, 52)
        a = wh.mdot(x, wh.apply_S(y))[0]
        b = wh.mdot(y, wh.apply_S(x))[0]
        assert abs(a - b) <= 1e-5 * math.sqrt(wh.mdot(x, x)[0] * wh.mdot(y, y)[0])
    node = (p.n[0] - 7, p.n[1] - 2)
    want = window_sample(p, nt, v, node, reach=4)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    gv = np.array([got[c * nn + idx[node[1], node[0]]] for c in range(2)])
    assert np.abs(gv - want).max() <= tol32(nt) * np.abs(got).max(), (gv, want)
