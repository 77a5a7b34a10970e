"""Curvilinear 2D grids (Section 4.1, curvilinear form) on the GPU against the
oracle: metric terms from the SBP derivative of the mapping, the four
J-weighted fluxes, the mass rho J H h^2 and the mapped time-step bound."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import TOL64, oracle_all_rhs, rel_err, to_np, tol32, window_sample

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D, F = inputs.DIRICHLET, inputs.FREE


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


MAPS = {"annulus": inputs.annulus_mapping, "wavy": inputs.wavy_mapping,
        "identity": lambda n, h: np.meshgrid(np.arange(n[0]) * h, np.arange(n[1]) * h)}

# (mapping, interior nodes, bc, nrhs): ragged 32 x 8 tiles, every side type
CASES = [("annulus", [10, 9], [D, D, D, D], 1), ("annulus", [41, 13], [D, D, D, F], 2),
         ("wavy", [12, 35], [F, F, D, F], 1), ("wavy", [6, 6], [F, F, F, F], 1),
         ("identity", [9, 10], [F, D, D, F], 1), ("annulus", [130, 67], [F, D, D, D], 1)]
# the fused one-launch step and the stress + divergence pair
KERNELS = ["fused", "fused16", "split"]


def _ids(c):
    return "%s_%s_bc%s_r%d" % (c[0], "x".join(map(str, c[1])), "".join(map(str, c[2])), c[3])


def _problem(mapname, nu, bc, nrhs=1, seed=21, implicit=0, omega=None):
    p = inputs.small_problem(2, nu, 4, bc, seed=seed, nrhs=nrhs, omega=omega)
    p.mapping = MAPS[mapname](p.n, p.h)
    p.implicit = implicit
    return p


def _wh(p, precision="fp64", nt=0):
    from paper_2205_12344_gb300.api import WaveHoltz
    return WaveHoltz(p, precision=precision, nt=nt)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_mapped_setup_and_operator_match_oracle(case, kernel, monkeypatch):
    monkeypatch.setenv("EWH_CURV", kernel)
    mapname, nu, bc, nrhs = case
    p = _problem(mapname, nu, bc, nrhs)
    s = O.build_system(p)
    with _wh(p) as wh:
        assert wh.info.nt == s.nt
        assert abs(wh.info.kt - s.kt) <= 1e-14 * s.kt
        u = inputs.random_vectors(p, 1, 5)[0]
        got = to_np(wh.apply_minvK(u))
    want = oracle_all_rhs(s, lambda ss, x, r: O.minv_K(ss, x), u)
    assert rel_err(got, want) < 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_mapped_S_and_Pi0_match_oracle(case, kernel, monkeypatch):
    monkeypatch.setenv("EWH_CURV", kernel)
    mapname, nu, bc, nrhs = case
    p = _problem(mapname, nu, bc, nrhs)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 7)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(p.nrhs)])
    with _wh(p) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
    assert rel_err(got, want) < TOL64
    assert rel_err(got0, want0) < TOL64
    with _wh(p, "fp32") as wh:
        got32 = to_np(wh.apply_S(v))
        got64 = to_np(wh.apply_S(v, fp64=True))
    assert rel_err(got32, want) < tol32(s.nt), rel_err(got32, want)
    assert rel_err(got64, want) < TOL64


def test_mapped_autotuner_picks_a_mapped_kernel(monkeypatch):
    """The autotuner times the two mapped kernels (never a Cartesian variant
    cached for the same grid size) and the pick matches the oracle."""
    from paper_2205_12344_gb300 import _lib as L
    monkeypatch.delenv("EWH_CURV", raising=False)
    p = _problem("wavy", [70, 40], [D, D, D, F])
    s = O.build_system(p)
    with _wh(p, "fp32") as wh:
        got0 = to_np(wh.apply_Pi0())
        variant = L.ewh_get_info(wh.ctx).kernel_variant[1]
    assert variant in (0, 1)
    assert rel_err(got0, O.apply_Pi0(s)) < tol32(s.nt)


def test_mapped_identity_is_the_cartesian_path():
    """x = q, y = r through the mapped kernels gives the Cartesian result."""
    p = _problem("identity", [37, 11], [F, D, D, F], nrhs=2)
    v = inputs.random_vectors(p, 1, 3)[0]
    with _wh(p) as wh:
        a = to_np(wh.apply_S(v))
        a0 = to_np(wh.apply_Pi0())
        nt = wh.info.nt
    p.mapping = None
    with _wh(p) as wh:
        assert wh.info.nt == nt
        b = to_np(wh.apply_S(v))
        b0 = to_np(wh.apply_Pi0())
    assert rel_err(a, b) < 1e-12 and rel_err(a0, b0) < 1e-12


# omega away from every discrete eigenfrequency: min(1 - beta) is 7e-4 and 4e-4
# over the spectrum of S (a frequency next to one leaves I - S indefinite)
@pytest.mark.parametrize("mapname,omega", [("annulus", 14.0), ("wavy", 15.5)])
def test_mapped_solves_reach_direct_solution(mapname, omega):
    p = _problem(mapname, [22, 17], [D, F, D, D], omega=omega)
    s = O.build_system(p)
    v = O.helmholtz_direct(s)
    with _wh(p) as wh:
        for method in ("solve", "solve_minres"):
            x, info = getattr(wh, method)(tol=1e-11, maxit=2000)
            assert info.status == 0 and info.rel_res <= 1e-11
            assert np.linalg.norm(to_np(x) - v) <= 1e-8 * np.linalg.norm(v)
    with _wh(p, "fp32") as wh:
        x, info = wh.solve(tol=1e-8, maxit=2000)
    assert info.status == 0 and info.rel_res <= 1e-8
    assert np.linalg.norm(to_np(x) - v) <= 1e-5 * np.linalg.norm(v)


def test_mapped_implicit_scheme_matches_oracle():
    p = _problem("annulus", [12, 10], [F, D, D, F], implicit=1)
    s = O.build_system(p, nt=8)
    v = inputs.random_vectors(p, 1, 9)[0]
    with _wh(p, nt=8) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
    assert rel_err(got, O.apply_S(s, v)) < 1e-10
    assert rel_err(got0, O.apply_Pi0(s)) < 1e-10


def test_mapped_rejections():
    from paper_2205_12344_gb300._lib import EwhError
    p = _problem("annulus", [10, 9], [D, D, D, D])
    X, Y = p.mapping
    p.mapping = (-X, Y)                       # reflected: J < 0 everywhere
    with pytest.raises(EwhError, match="J <= 0"):
        _wh(p)
    q = inputs.small_problem(2, [10, 9], 2, [D, D, D, D], seed=1)
    q.mapping = inputs.annulus_mapping(q.n, q.h)
    with pytest.raises(EwhError, match="order 4"):
        _wh(q)
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    with pytest.raises(ValueError):
        WaveHoltzBatch([_problem("wavy", [8, 8], [D, D, D, D])])


# ---------------------------------------------------------------- full size

def _sector_1024():
    """The layered 1024^2 workload mapped onto an annular sector of about the
    same extent (radius 1.5 L .. 2.5 L along q, 0.5 rad along r)."""
    p = inputs.cfg_layered_2d(nu=1024, order=4)
    L = (p.n[0] - 1) * p.h
    p.mapping = inputs.annulus_mapping(p.n, p.h, span=0.5, r0=1.5 * L, dr=L)
    return p


@pytest.mark.parametrize("prec,node", [("fp32", "top_left"), ("fp64", "bottom_right")])
def test_mapped_sector_1024_sampled_parity(prec, node, monkeypatch):
    """The mapped bench workload at full size, in the kernel the autotuner
    picks: S v at a node near a corner from the oracle on its domain of
    dependence (the window keeps the node coordinates, so its metric terms
    equal the full grid's away from the window's own sides)."""
    import math
    monkeypatch.delenv("EWH_CURV", raising=False)
    p = _sector_1024()
    from paper_2205_12344_gb300.api import WaveHoltz
    with WaveHoltz(p, precision=prec) as wh:
        nt = wh.info.nt
        v = inputs.random_vectors(p, 1, 31)[0]
        got = to_np(wh.apply_S(v))
    dtc = O.cfl_dt_mapped(p.n, p.h, p.cfl, p.rho, p.lam, p.mu, *p.mapping)
    assert nt == max(5, int(math.ceil(2 * math.pi / p.omega / dtc)))
    xy = (6, p.n[1] - 2) if node == "top_left" else (p.n[0] - 3, 4)
    want = window_sample(p, nt, v, xy, reach=4)
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    gv = np.array([got[c * nn + idx[xy[1], xy[0]]] for c in range(2)])
    tol = tol32(nt) if prec == "fp32" else TOL64
    assert np.abs(gv - want).max() <= tol * np.abs(got).max(), (gv, want)
