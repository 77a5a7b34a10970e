"""The fused 3D order-4 FP32 step (one launch per leapfrog level marching
along z: bulk-tensor u planes, stresses on chip) against the oracle: S and
Pi 0 (Section 3, eq. qoper; the leapfrog of Section 4.3 with the order-4 SBP
operator of Section 4.1) on grids with several tiles, ragged tails, every side
type, z ranges split across CTAs, and several right-hand sides; the 256^3
random-field workload node by node (N_t = 6 windows) and as a whole against
the per-level kernel pair; and the bounded mbarrier wait.

EWH_STEP3D_O4=zm16|zm8|pair selects the kernel (32 x 16 or 32 x 8 tiles, or
the per-level pair); EWH_ZM_GRID caps the persistent grid so that each CTA
walks long (tile, z range) shares.
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


def _launches_per_apply(wh, v):
    """Kernel launches of one S apply (pack + levels + unpack)."""
    a = wh.kernel_launches()
    wh.apply_S(v)
    return wh.kernel_launches() - a


# (unknown-ish nodes per axis, sides, right-hand sides, grid cap)
CASES = [([70, 22, 12], [D, D, D, D, D, D], 2, 0),     # 3 x 2 tiles, ragged in x and y
         ([72, 24, 12], [F, F, F, F, F, F], 1, 0),     # every side free: closures and boundary terms
         ([70, 22, 12], [D, F, F, D, D, F], 1, 5),     # 5 CTAs: long shares crossing tiles
         ([33, 17, 16], [D, D, D, D, F, D], 2, 3),     # one-column / one-row last tiles at Dirichlet sides
         ([40, 40, 30], [D, D, D, F, F, D], 1, 7),
         # last tiles of 4 (Dirichlet) and 5 / 3 / 1 (free) unknowns: the stencils of the tile
         # before them would reach past its staged tiles, so the tile origins shift
         ([36, 20, 14], [D, D, D, D, D, F], 1, 0),
         ([36, 18, 14], [D, F, D, F, F, D], 1, 0),
         ([32, 16, 13], [D, F, D, F, D, D], 2, 4)]


def _unknowns(p, bc, a):
    return p.n[a] - (bc[2 * a] == D) - (bc[2 * a + 1] == D)


@pytest.mark.parametrize("shape", ["zm16", "zm8"])
@pytest.mark.parametrize("nu,bc,nrhs,cap", CASES, ids=lambda c: str(c))
def test_zmarch_S_and_Pi0_match_oracle(nu, bc, nrhs, cap, shape, monkeypatch):
    monkeypatch.setenv("EWH_STEP3D_O4", shape)
    if cap:
        monkeypatch.setenv("EWH_ZM_GRID", str(cap))
    p = inputs.small_problem(3, nu, 4, bc, seed=61, nrhs=nrhs)
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 62)[0]
    want = oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)
    want0 = np.concatenate([O.apply_Pi0(s, r) for r in range(p.nrhs)])
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        got0 = to_np(wh.apply_Pi0())
        # one launch per level (the per-level pair takes two), plus pack and unpack
        assert _launches_per_apply(wh, v) == s.nt + 2
        again = to_np(wh.apply_S(v))
    assert rel_err(got, want) < tol32(s.nt)
    assert rel_err(got0, want0) < tol32(s.nt)
    assert np.array_equal(again, got)                  # deterministic: no read of a plane in flight


def test_zmarch_solve_reaches_oracle_residual(monkeypatch):
    """The mixed-precision CG on the fused FP32 operator reaches a residual
    the oracle confirms in FP64 (eq. amat_sym)."""
    monkeypatch.setenv("EWH_STEP3D_O4", "zm")
    p = inputs.small_problem(3, [24, 20, 14], 4, [D, D, D, D, D, F], seed=65, omega=6.0)
    s = O.build_system(p)
    with _fp32(p) as wh:
        x, info = wh.solve(tol=1e-7, maxit=2000)
    assert info.status == 0 and info.rel_res <= 1e-7
    x = to_np(x)
    b = O.apply_Pi0(s)
    r = b - (x - O.apply_S(s, x))
    assert math.sqrt(O.mdot(s, r, r) / O.mdot(s, b, b)) <= 1.01e-7


@pytest.fixture(scope="module")
def grf256_nt6():
    """The 256^3 random-field workload with w raised so that N_t = 6."""
    p = inputs.cfg_grf_3d(nu=256, order=4)
    dtc = O.cfl_dt(3, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    p.omega = 2 * math.pi / (5.5 * dtc)
    v = inputs.random_vectors(p, 1, 81)[0]
    return p, v


@pytest.mark.parametrize("shape", ["zm16", "zm8"])
def test_zmarch_256_sampled_nodes(grf256_nt6, shape, monkeypatch):
    """S v of the fused kernel on the 256^3 workload at nodes in the
    interior, on tile seams in x and y, next to each side and in a corner,
    against the oracle on each node's domain of dependence."""
    monkeypatch.setenv("EWH_STEP3D_O4", shape)
    p, v = grf256_nt6
    with _fp32(p) as wh:
        got = to_np(wh.apply_S(v))
        assert wh.info.nt == 6
        assert _launches_per_apply(wh, v) == 6 + 2
    n = p.n[0]
    nodes = [(129, 131, 127), (32, 70, 100), (33, 70, 100), (140, 16, 90), (140, 17, 90),
             (1, 100, 120), (n - 2, 90, 60), (80, 2, 40), (90, n - 3, 200), (100, 110, 1), (60, 50, n - 4),
             (2, 3, 1), (n - 2, n - 2, n - 2)]
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    scale = np.abs(got).max()
    for node in nodes:
        x, y, z = node
        g = np.array([got[c * nn + idx[z, y, x]] for c in range(3)])
        want = window_sample(p, 6, v, node, reach=4)
        assert np.abs(g - want).max() <= tol32(6) * scale, (node, g, want)


def test_zmarch_256_whole_field_matches_pair(grf256_nt6, monkeypatch):
    """Every node of the 256^3 fused S v (both tile shapes) against the
    per-level pair (whose small-grid parity with the oracle is tested above
    and in test_gpu_parity)."""
    p, v = grf256_nt6
    monkeypatch.setenv("EWH_STEP3D_O4", "pair")
    with _fp32(p) as wh:
        a = to_np(wh.apply_S(v))
    for shape in ("zm16", "zm8"):
        monkeypatch.setenv("EWH_STEP3D_O4", shape)
        with _fp32(p) as wh:
            b = to_np(wh.apply_S(v))
        assert rel_err(b, a) < 2 * tol32(6), shape


def test_zmarch_wait_gives_up_and_recovers(monkeypatch):
    """A zero wait limit makes every mbarrier wait give up: the accumulator
    comes back NaN, the give-ups are counted, and with the limit restored the
    same context returns the same S v as before."""
    monkeypatch.setenv("EWH_STEP3D_O4", "zm")
    p = inputs.small_problem(3, [70, 22, 12], 4, [D, F, F, D, D, F], seed=66)
    v = inputs.random_vectors(p, 1, 67)[0]
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
