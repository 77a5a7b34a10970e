"""The on-chip resident wave solve (2D, order-4 SBP, FP32 stencil, one
right-hand side: every leapfrog level of S in one cooperative launch, the
state in shared memory and registers, halos exchanged through global memory
at one grid barrier per level) against the oracle.

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


def test_resident_not_used_for_batches_or_several_rhs(monkeypatch):
    """Batch members (concurrent graph branches) and multi-rhs contexts keep
    the per-level kernels."""
    monkeypatch.setenv("EWH_STEP2D_O4", "r0")
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    p2 = inputs.small_problem(2, [30, 30], 4, [D, D, D, F, 0, 0], seed=45, nrhs=2)
    s2 = O.build_system(p2)
    v2 = inputs.random_vectors(p2, 1, 46)[0]
    with _fp32(p2) as wh:
        got = to_np(wh.apply_S(v2))
        assert _variant(wh) < VARIANT_RESIDENT
    want = oracle_all_rhs(s2, lambda ss, x, r: O.apply_S(ss, x, r), v2)
    assert rel_err(got, want) < tol32(s2.nt)
    probs = [inputs.small_problem(2, [30, 30], 4, [D, D, D, F, 0, 0], seed=47 + k) for k in range(2)]
    b = WaveHoltzBatch(probs, precision="fp32")
    try:
        b.solve(tol=1e-6, maxit=20, raise_on_error=False)
        for k in range(2):
            ctx = L.ewh_batch_member(b.b, k)
            assert L.ewh_get_info(ctx).kernel_variant[1] < VARIANT_RESIDENT
    finally:
        b.close()


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
