"""Plant plausible mistakes in (copies of) the oracle, on the CPU, and check
that the pins catch each one: a wrong sign in the Taylor start, a dropped
-1/4 filter shift, a mixed term with the wrong sign, the uncorrected time
step used where the corrected one is meant, and, on mapped grids, a metric
term with the wrong sign, two metric terms transposed, or the Jacobian left
out."""
import math

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs


def _fixed_point_residual(s):
    v = O.helmholtz_direct(s)
    return np.linalg.norm(O.apply_Pi(s, v) - v) / np.linalg.norm(v)


def _prob():
    return inputs.small_problem(2, [8, 9], 2, [0, 0, 0, 1], seed=7)


def test_planted_start_sign_is_caught(monkeypatch):
    s = O.build_system(_prob())
    assert _fixed_point_residual(s) < 1e-12
    orig = O.minv_K
    calls = {"n": 0}

    def wrong_first_call(sys_, u):            # the first M^{-1}K call builds u^{-1}
        calls["n"] += 1
        out = orig(sys_, u)
        return -out if calls["n"] == 1 else out

    monkeypatch.setattr(O, "minv_K", wrong_first_call)
    assert _fixed_point_residual(s) > 1e-6


def test_planted_filter_shift_is_caught():
    w = O.filter_weights(50, 1)
    nvec = np.arange(51)
    eta = np.ones(51)
    eta[0] = eta[-1] = 0.5
    wrong = (2.0 / 50) * eta * np.cos(2 * np.pi * nvec / 50)      # -1/4 dropped
    assert abs(w.sum() + 0.5) < 1e-13
    assert abs(wrong.sum() + 0.5) > 0.1


def test_planted_mixed_sign_is_caught(monkeypatch):
    p = inputs.small_problem(2, [7, 8], 2, [1, 1, 1, 1], seed=5)
    orig = O.centred_difference

    def flipped(N):
        return -orig(N) if N == p.n[1] else orig(N)   # flip only the y difference

    K, *_rest = O.assemble(2, p.n, p.h, 2, p.bc, p.rho, p.lam, p.mu)
    monkeypatch.setattr(O, "centred_difference", flipped)
    Kw, Md, Wd, rho, sel = O.assemble(2, p.n, p.h, 2, p.bc, p.rho, p.lam, p.mu)
    xs = inputs._coords(p.n, p.h)
    nn = len(sel)
    rot = np.concatenate([-xs[1].reshape(-1)[sel], xs[0].reshape(-1)[sel]])
    assert np.abs(K @ rot).max() < 1e-12 * abs(K).max()
    assert np.abs(Kw @ rot).max() > 1e-3 * abs(Kw).max() * p.h


def test_planted_uncorrected_step_is_caught():
    p = _prob()
    s = O.build_system(p)
    s.kt = s.dt ** 2                             # c dropped while v solves the w problem
    assert _fixed_point_residual(s) > 1e-6


# ---------------------------------------------------------------- mapped grids

def _sector_interior_error(m=33):
    """Max error of -M^{-1} K u against the hand-written elastic operator at
    nodes 9 or more from every side of an annular-sector grid (lambda = 2,
    mu = 1, rho = 1)."""
    n = [m, m]
    h = 1.0 / (m - 1)
    X, Y = inputs.annulus_mapping(n, h)
    ones = np.ones((m, m))
    K, M, W, rho_u, sel = O.assemble_mapped(n, h, [1, 1, 1, 1], ones, 2.0 * ones, ones, X, Y)
    x, y = X.reshape(-1)[sel], Y.reshape(-1)[sel]
    u = np.concatenate([0.3 * np.sin(x) * np.cos(y), 0.2 * np.cos(2 * x) * np.sin(y)])
    got = -(K @ u) / M
    dxdiv = -0.3 * np.sin(x) * np.cos(y) - 0.4 * np.sin(2 * x) * np.cos(y)
    dydiv = -0.3 * np.cos(x) * np.sin(y) - 0.2 * np.cos(2 * x) * np.sin(y)
    ex = 3.0 * dxdiv - 0.6 * np.sin(x) * np.cos(y)
    ey = 3.0 * dydiv - 1.0 * np.cos(2 * x) * np.sin(y)
    ii, jj = np.meshgrid(np.arange(m), np.arange(m))
    inner = ((ii >= 9) & (ii <= m - 10) & (jj >= 9) & (jj <= m - 10)).reshape(-1)[sel]
    nn = len(sel)
    return max(np.abs(got[:nn] - ex)[inner].max(), np.abs(got[nn:] - ey)[inner].max())


@pytest.mark.parametrize("plant", ["rx_sign", "qy_for_ry", "no_jacobian"])
def test_planted_metric_mistakes_are_caught(plant, monkeypatch):
    """A wrong sign in a metric term, a transposed metric term, or the
    Jacobian left out of the weights and mass: the sector truncation pin
    (fourth-order interior accuracy) fails for each."""
    good = _sector_interior_error()
    assert good < 1e-4
    orig = O.mapped_metrics

    def planted(n, h, X, Y):
        J, qx, qy, rx, ry = orig(n, h, X, Y)
        if plant == "rx_sign":
            return J, qx, qy, -rx, ry
        if plant == "qy_for_ry":
            return J, qx, ry, rx, qy
        return np.ones_like(J), qx, qy, rx, ry

    monkeypatch.setattr(O, "mapped_metrics", planted)
    assert _sector_interior_error() > 100 * good
