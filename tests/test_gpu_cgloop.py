"""CG iterations under device control: a while-conditional graph node runs
the iterations (the leapfrog levels of the S apply, the Krylov kernels, then
a control kernel that decides whether the host must act), and the host polls
once per window of EWH_CG_POLL iterations instead of after every iteration.
The decisions are the host loop's (FP64 residual replacement when a residual
reached tol or fell by the drop factor, breakdown, the iteration limit), taken
from the same scalars, so iterates, iteration counts and residual histories
must equal the host-driven loop's (EWH_CG_POLL=1) bit for bit; CG in the M
inner product on (I - S) v = Pi 0 (Section 3, eq. amat_sym).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2205_12344_gb300 import inputs
from _helpers import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D, F = inputs.DIRICHLET, inputs.FREE


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _solve(p, precision, window, monkeypatch, tol, maxit, env=None):
    from paper_2205_12344_gb300.api import WaveHoltz
    monkeypatch.setenv("EWH_CG_POLL", str(window))
    for k, v in (env or {}).items():
        monkeypatch.setenv(k, v)
    with WaveHoltz(p, precision=precision) as wh:
        x, info = wh.solve(tol=tol, maxit=maxit, raise_on_error=False)
        hist = list(wh.residual_history())
        launches = wh.kernel_launches()
    return to_np(x), info, hist, launches


CASES = [("fp64", [40, 34], [D, D, D, F], 1, {}),
         ("fp32", [40, 34], [D, D, D, F], 1, {}),                          # residual replacements
         ("fp32", [70, 34], [D, D, D, F], 3, {"EWH_STEP2D_O4": "split"}),   # rhs converging apart
         ("fp32", [40, 34], [D, D, D, F], 2, {"EWH_STEP2D_O4": "r0"}),      # resident launches in the body
         ("fp32", [70, 34], [D, D, D, F], 2, {"EWH_STEP2D_O4": "ym"})]


@pytest.mark.parametrize("precision,grid,bc,nrhs,env", CASES, ids=lambda c: str(c))
@pytest.mark.parametrize("window", [32, 7])
def test_device_loop_equals_host_loop(precision, grid, bc, nrhs, env, window, monkeypatch):
    p = inputs.small_problem(2, grid, 4, bc, seed=42, nrhs=nrhs, omega=6.0)
    xh, ih, hh, lh = _solve(p, precision, 1, monkeypatch, 1e-9, 5000, env)
    xd, idv, hd, ld = _solve(p, precision, window, monkeypatch, 1e-9, 5000, env)
    assert ih.status == 0 and idv.status == 0
    assert idv.iters == ih.iters and idv.s_applies == ih.s_applies and idv.s_applies_fp64 == ih.s_applies_fp64
    assert np.array_equal(xd, xh)
    assert hd == hh
    # the same kernels ran: the control kernel once per iteration on top
    assert ld == lh + idv.iters


def test_device_loop_stops_at_maxit(monkeypatch):
    """An iteration limit that is no multiple of the window: the last window
    is cut to the limit; status 'not converged', the same iterate as the host
    loop after the same number of iterations."""
    p = inputs.small_problem(2, [70, 34], 4, [D, D, D, F], seed=42, nrhs=1, omega=6.0)
    xh, ih, hh, _ = _solve(p, "fp64", 1, monkeypatch, 1e-14, 11)
    xd, idv, hd, _ = _solve(p, "fp64", 4, monkeypatch, 1e-14, 11)
    assert ih.iters == 11 and idv.iters == 11 and idv.status == ih.status != 0
    assert np.array_equal(xd, xh) and hd == hh
