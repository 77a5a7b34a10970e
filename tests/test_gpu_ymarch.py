"""The fused 2D order-4 FP32 step (one launch per leapfrog level marching
along y: one warp per strip of 60 columns, bulk-tensor u rows, stresses on
chip) against the oracle: S and Pi 0 (Section 3, eq. qoper; the leapfrog of
Section 4.3 with the order-4 SBP operator of Section 4.1) on grids with
several strips, ragged tails, every side type, row ranges split across CTAs
and several right-hand sides; a batch member's size as a whole against the
per-level split kernels; batches whose members run it; and the bounded
mbarrier wait.

EWH_STEP2D_O4=ym selects the kernel; EWH_YM_ROWS sets the least number of
rows per CTA share (1: many short shares, a large value: one CTA walks every
strip and right-hand side).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import oracle_all_rhs, rel_err, to_np, tol32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D, F = inputs.DIRICHLET, inputs.FREE
YM_VARIANT = 8


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


def _launches_per_apply(wh, v):
    a = wh.kernel_launches()
    wh.apply_S(v)
    return wh.kernel_launches() - a


# (grid nodes per axis - 2, sides x-lo x-hi y-lo y-hi, right-hand sides, rows per share)
CASES = [([128, 38], [D, D, D, D], 2, 0),      # 3 strips, ragged last strip
         ([122, 34], [F, F, F, F], 1, 1),      # every side free; shares of one or two rows
         ([60, 48], [D, F, F, D], 3, 10 ** 6),  # one CTA walks every strip and rhs
         ([62, 30], [D, D, D, F], 1, 7),       # 62 unknowns along x: last strip of 2 -> shifted
         ([124, 10], [D, D, F, D], 2, 3),      # 124 unknowns (last strip 4 -> shifted); 12 nodes along y
         ([62, 13], [D, F, D, F], 1, 5),       # 63 unknowns, free x-high: last strip 3 -> shifted
         ([120, 20], [D, F, F, F], 1, 0),      # 121 unknowns, free x-high: last strip 1 -> shifted
         ([121, 25], [F, F, D, D], 2, 2),      # 123 unknowns: last strip 3 -> shifted
         ([123, 14], [F, F, F, D], 1, 4)]      # 125 unknowns: last strip 5 -> shifted


@pytest.mark.parametrize("nu,bc,nrhs,rows", CASES, ids=lambda c: str(c))
def test_ymarch_S_and_Pi0_match_oracle(nu, bc, nrhs, rows, monkeypatch):
    monkeypatch.setenv("EWH_STEP2D_O4", "ym")
    if rows:
        monkeypatch.setenv("EWH_YM_ROWS", str(rows))
    p = inputs.small_problem(2, nu, 4, bc, seed=71, nrhs=nrhs)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 72)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(p.nrhs)])
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
        assert _variant(wh) == YM_VARIANT
        # one launch per level, plus pack and unpack
        assert _launches_per_apply(wh, v) == s.nt + 2
        again = to_np(wh.apply_S(v))
    assert rel_err(got, want) < tol32(s.nt)
    assert rel_err(got0, want0) < tol32(s.nt)
    assert np.array_equal(again, got)  # deterministic: no read of a row in flight


def test_ymarch_solve_reaches_oracle_residual(monkeypatch):
    """The mixed-precision CG on the fused FP32 operator reaches a residual
    the oracle confirms in FP64 (eq. amat_sym)."""
    monkeypatch.setenv("EWH_STEP2D_O4", "ym")
    p = inputs.small_problem(2, [70, 34], 4, [D, D, D, F], seed=42, nrhs=2, omega=6.0)
    s = O.build_system(p)
    with _fp32(p) as wh:
        x, info = wh.solve(tol=1e-7, maxit=5000)
        assert _variant(wh) == YM_VARIANT
    assert info.status == 0 and info.rel_res <= 1e-7
    x = to_np(x)
    n = s.K.shape[0]
    for r in range(p.nrhs):
        b = O.apply_Pi0(s, r)
        xr = x[r * n:(r + 1) * n]
        res = b - (xr - O.apply_S(s, xr, r))
        assert math.sqrt(O.mdot(s, res, res) / O.mdot(s, b, b)) <= 1.01e-7


def test_ymarch_member_size_whole_field_matches_split(monkeypatch):
    """Every node of S v at a batch member's size (layered 256^2, 4 shots)
    against the oracle-checked per-level split kernels."""
    p = inputs.cfg_layered_2d(nu=256, order=4, nrhs=4, shot_x=[0.5, 1.0, 1.5, 2.0])
    v = inputs.random_vectors(p, 1, 73)[0]
    monkeypatch.setenv("EWH_STEP2D_O4", "split")
    with _fp32(p) as wh:
        a = to_np(wh.apply_S(v))
        nt = wh.info.nt
    monkeypatch.setenv("EWH_STEP2D_O4", "ym")
    with _fp32(p) as wh:
        b = to_np(wh.apply_S(v))
        assert _variant(wh) == YM_VARIANT
    assert rel_err(b, a) < 2 * tol32(nt)


def test_ymarch_batch_members_equal_single(monkeypatch):
    """Batch members that run the y-march return the same S v as the same
    problems alone (same kernels, same order: bitwise)."""
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    monkeypatch.setenv("EWH_STEP2D_O4", "ym")
    probs = [inputs.small_problem(2, [70, 40], 4, [D, D, D, F], seed=74, nrhs=2),
             inputs.small_problem(2, [130, 50], 4, [D, D, D, F], seed=75, nrhs=1)]
    vs = [inputs.random_vectors(p, 1, 76 + k)[0] for k, p in enumerate(probs)]
    with WaveHoltzBatch(probs, "fp32") as wb:
        outs = [to_np(o) for o in wb.apply_S(vs)]
    for p, v, o in zip(probs, vs, outs):
        with _fp32(p) as wh:
            single = to_np(wh.apply_S(v))
            assert _variant(wh) == YM_VARIANT
        assert np.array_equal(o, single)
        s = O.build_system(p)
        assert rel_err(o, oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)) < tol32(s.nt)


def test_ymarch_wait_gives_up_and_recovers(monkeypatch):
    """A zero wait limit makes every mbarrier wait give up: the accumulator
    comes back NaN, the give-ups are counted, and with the limit restored the
    same context returns the same S v as before."""
    monkeypatch.setenv("EWH_STEP2D_O4", "ym")
    p = inputs.small_problem(2, [128, 38], 4, [D, F, F, D], seed=77, nrhs=2)
    v = inputs.random_vectors(p, 1, 78)[0]
    with _fp32(p) as wh:
        good = to_np(wh.apply_S(v))
        wh.reset_stats()
        wh.set_grid_wait(0)
        bad = to_np(wh.apply_S(v))
        assert np.isnan(bad).all()
        assert wh.stats().grid_wait_timeouts >= 1
        wh.set_grid_wait(10 ** 9)
        again = to_np(wh.apply_S(v))
    assert np.array_equal(again, good)
