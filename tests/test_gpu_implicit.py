"""The implicit time-corrected scheme (Section 4.4) on the GPU against the
oracle: every level solves with I + (dt^2/2) M^{-1} K by an inner CG in the
M inner product on the device (FP64)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import oracle_all_rhs, rel_err, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D, F = inputs.DIRICHLET, inputs.FREE
TOL_IMPLICIT = 1e-10   # FP64 levels, each solved to a relative 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _implicit(dim, nu, order, bc, nt, corrected=1, seed=5, nrhs=1, omega=None):
    p = inputs.small_problem(dim, nu, order, bc + [0] * (6 - len(bc)), seed=seed, nrhs=nrhs, omega=omega)
    p.implicit = 1
    p.corrected = corrected
    return p, O.build_system(p, nt=nt)


def _wh(p, nt):
    from paper_2205_12344_gb300.api import WaveHoltz
    return WaveHoltz(p, precision="fp64", nt=nt)


CASES = [(2, [9, 8], 2, [D, D, D, F], 6, 1), (2, [12, 10], 4, [F, D, D, F], 10, 1),
         (2, [9, 8], 2, [D, F, F, D], 7, 0), (3, [5, 6, 5], 2, [D, D, D, D, D, F], 6, 1)]


@pytest.mark.parametrize("dim,nu,order,bc,nt,corrected", CASES)
def test_implicit_S_and_Pi0_match_oracle(dim, nu, order, bc, nt, corrected):
    p, s = _implicit(dim, nu, order, bc, nt, corrected, nrhs=2)
    v = inputs.random_vectors(p, 1, 61)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(p.nrhs)])
    with _wh(p, nt) as wh:
        assert wh.info.nt == nt
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
    assert rel_err(got, want) < TOL_IMPLICIT
    assert rel_err(got0, want0) < TOL_IMPLICIT


@pytest.mark.parametrize("method", ["solve", "solve_cr", "solve_minres"])
def test_implicit_solves_reach_helmholtz_solution(method):
    """With the modified alpha the fixed point is the w problem itself."""
    p, s = _implicit(2, [10, 9], 2, [D, D, D, F], 8)
    v = O.helmholtz_direct(s)
    with _wh(p, 8) as wh:
        x, info = getattr(wh, method)(tol=1e-10, maxit=400)
    assert info.status == 0 and info.rel_res <= 1e-10
    assert np.linalg.norm(to_np(x) - v) <= 1e-7 * np.linalg.norm(v)


def test_implicit_indefinite_system_minres():
    """Five implicit steps per period make M(I - S) indefinite (the oracle
    pins that with the dense S); GPU MINRES reaches the Helmholtz solution with
    a non-increasing residual (the Section 4.4 remark)."""
    p, s = _implicit(2, [6, 5], 2, [D, F, D, D], 5, seed=3, omega=7.5)
    v = O.helmholtz_direct(s)
    with _wh(p, 5) as wh:
        x, info = wh.solve_minres(tol=1e-11, maxit=500)
        hist = wh.residual_history()
    assert info.status == 0
    assert np.all(np.diff(hist) <= 1e-12)
    assert np.linalg.norm(to_np(x) - v) <= 1e-8 * np.linalg.norm(v)


def test_implicit_rejections():
    """FP32 precision, a missing nt and batch membership are rejected."""
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz, WaveHoltzBatch
    p, _ = _implicit(2, [9, 8], 2, [D, D, D, F], 6)
    with pytest.raises(L.EwhError) as e:
        WaveHoltz(p, precision="fp32", nt=6)
    assert e.value.status == L.EWH_EINVAL
    with pytest.raises(L.EwhError) as e:
        WaveHoltz(p, precision="fp64", nt=0)
    assert e.value.status == L.EWH_EINVAL
    with pytest.raises(L.EwhError) as e:
        WaveHoltzBatch([p], precision="fp64")
    assert e.value.status == L.EWH_EINVAL
