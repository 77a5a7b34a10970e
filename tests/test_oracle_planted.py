"""Plant plausible mistakes in (copies of) the oracle, on the CPU, and check
that the pins catch each one: a wrong sign in the Taylor start, a dropped
-1/4 filter shift, a mixed term with the wrong sign, and the uncorrected
time step used where the corrected one is meant."""
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
