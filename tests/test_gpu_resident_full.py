"""The on-chip resident wave solve on the full 1024^2 layered workload, node by
node: every register slot of the regular node pairs, both sides of CTA seams,
the narrower edge-column blocks and the special (SBP closure, boundary-term,
Dirichlet-neighbour) nodes by every side type, against the oracle on each
node's domain of dependence (S of Section 3 with the trapezoid rule of eq.
qoper, the leapfrog of Section 4.3).  Also the whole 1024^2 field against the
per-level split kernels, the FP64 split kernels against the oracle at 1e-10,
and the bounded grid-barrier wait: a zero limit makes every wait give up, the
apply returns NaN, the solve finishes on the FP64 operator and the context
stays usable.

The frequency is raised so that N_t = 6 (windows of radius (6+2)*4 = 32
nodes); the grid, medium, boundary conditions, kernel and CTA partition are
those of the benchmark workload.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import rel_err, to_np, tol32, window_sample

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


@pytest.fixture(scope="module")
def layered_nt6():
    """The layered 1024^2 workload with w raised so that N_t = 6, and one
    random input vector."""
    p = inputs.cfg_layered_2d(nu=1024, order=4)
    dtc = O.cfl_dt(2, 4, p.h, p.cfl, p.rho, p.lam, p.mu)
    p.omega = 2 * math.pi / (5.5 * dtc)
    v = inputs.random_vectors(p, 1, 71)[0]
    return p, v


def _blocks(plan, n0, n1):
    """CTA blocks (cx, cy, X0, Y0, wx, wy) of a resident partition
    (shape, px, py, bx, ex, by, threads, pairs)."""
    _, px, py, bx, ex, by, _, _ = plan
    out = []
    for cy in range(py):
        for cx in range(px):
            X0 = 0 if cx == 0 else ex + (cx - 1) * bx
            wx = ex if cx == 0 else min(bx, n0 - X0)
            Y0 = cy * by
            out.append((cx, cy, X0, Y0, wx, min(by, n1 - Y0)))
    return out


def _rect(blk, n0, n1):
    """Regular rectangle [xa, xb) x [ya, yb) of a block (block-local; even
    width), or None: its nodes are done in pairs along x, pair l at
    (xa + 2 (l % (w/2)), ya + l // (w/2)), thread l % NT, register slot l // NT."""
    _, _, X0, Y0, wx, wy = blk
    xa, xb = max(0, 4 - X0), min(wx, n0 - 4 - X0)
    ya, yb = max(0, 4 - Y0), min(wy, n1 - 4 - Y0)
    if xb <= xa or yb <= ya:
        return None
    xb = xa + ((xb - xa) & ~1)
    return None if xb == xa else (xa, xb, ya, yb)


def _pair_node(blk, rect, l, second):
    _, _, X0, Y0, _, _ = blk
    xa, xb, ya, _ = rect
    w2 = (xb - xa) // 2
    return (X0 + xa + 2 * (l % w2) + second, Y0 + ya + l // w2)


def _owner(blocks, node):
    for b in blocks:
        if b[2] <= node[0] < b[2] + b[4] and b[3] <= node[1] < b[3] + b[5]:
            return b
    raise AssertionError("node %s in no block" % (node,))


def _slot_of(blocks, node, n0, n1, NT):
    """Register slot holding the node's filter accumulator, or None (special
    node: accumulator in shared memory)."""
    b = _owner(blocks, node)
    r = _rect(b, n0, n1)
    if r is None:
        return None
    jx, jy = node[0] - b[2], node[1] - b[3]
    xa, xb, ya, yb = r
    if not (xa <= jx < xb and ya <= jy < yb):
        return None
    l = (jy - ya) * ((xb - xa) // 2) + (jx - xa) // 2
    return l // NT


def _sample_nodes(plan, n0, n1):
    """Nodes covering every register slot of an interior block and of both
    edge-column blocks, both sides of an x seam and a y seam, and special
    nodes next to each side type (free top, Dirichlet bottom, left, right)."""
    _, px, py, _, _, _, NT, NP = plan
    blocks = _blocks(plan, n0, n1)
    nodes = []
    mid = [b for b in blocks if b[0] == px // 2 and b[1] == py // 2][0]
    for blk in (mid, [b for b in blocks if b[0] == 0 and b[1] == py // 2][0],
                [b for b in blocks if b[0] == px - 1 and b[1] == max(py // 2 - 1, 0)][0]):
        r = _rect(blk, n0, n1)
        npair = ((r[1] - r[0]) // 2) * (r[3] - r[2])
        for k in range(NP):
            if NT * k >= npair:
                break
            t = (37 * k + 11) % min(NT, npair - NT * k)
            nodes.append(_pair_node(blk, r, NT * k + t, k % 2))
    _, _, X0, Y0, wx, wy = mid
    ym, xm = Y0 + wy // 2, X0 + wx // 2
    nodes += [(X0 - 1, ym), (X0, ym), (xm, Y0 - 1), (xm, Y0)]            # seams
    nodes += [(xm, n1 - 1), (xm + 1, n1 - 3), (xm, 1), (xm - 1, 3)]      # free top, Dirichlet bottom
    nodes += [(1, ym), (3, ym + 1), (n0 - 2, ym), (n0 - 4, ym - 1)]      # Dirichlet left and right
    nodes += [(1, n1 - 1), (n0 - 2, 1)]                                  # corners
    return nodes, blocks


def _gather(p, vec, nodes):
    idx = inputs.unknown_index(p)
    nn = p.n_nodes()
    return np.array([[vec[c * nn + idx[y, x]] for c in range(2)] for (x, y) in nodes])


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_resident_1024_every_slot_and_seam(shape, layered_nt6, monkeypatch):
    """S v of the resident launch at nodes in every register slot, across CTA
    seams, in the edge-column blocks and at special nodes by every side type,
    each against the oracle on its domain of dependence (FP32 tolerance)."""
    from paper_2205_12344_gb300.api import WaveHoltz
    p, v = layered_nt6
    monkeypatch.setenv("EWH_STEP2D_O4", "r%d" % shape)
    with WaveHoltz(p, precision="fp32") as wh:
        got = to_np(wh.apply_S(v))
        from paper_2205_12344_gb300 import _lib as L
        info = L.ewh_get_info(wh.ctx)
        nt = info.nt
        plan = list(info.resident)[:8]
    assert nt == 6
    assert info.kernel_variant[1] == VARIANT_RESIDENT + shape and plan[0] == shape
    n0, n1 = p.n
    NT, NP = plan[6], plan[7]
    nodes, blocks = _sample_nodes(plan, n0, n1)
    # the sample reaches what it claims: every register slot of the interior
    # block, both sides of the seams, both edge-column blocks, special nodes
    slots = [_slot_of(blocks, nd, n0, n1, NT) for nd in nodes]
    assert set(s for s in slots if s is not None) == set(range(NP)), slots
    assert sum(s is None for s in slots) >= 10
    mid = [b for b in blocks if b[0] == plan[1] // 2 and b[1] == plan[2] // 2][0]
    assert _owner(blocks, nodes[-14]) != mid and _owner(blocks, nodes[-13]) == mid
    assert _owner(blocks, nodes[-12]) != mid and _owner(blocks, nodes[-11]) == mid
    assert any(_owner(blocks, nd)[0] == 0 for nd in nodes)
    assert any(_owner(blocks, nd)[0] == plan[1] - 1 for nd in nodes)
    gv = _gather(p, got, nodes)
    scale = np.abs(got).max()
    for nd, g in zip(nodes, gv):
        want = window_sample(p, nt, v, nd, reach=4)
        assert np.abs(g - want).max() <= tol32(nt) * scale, (nd, g, want)


def test_fp64_split_1024_sampled_nodes(layered_nt6):
    """The FP64 per-level kernels on the same workload and nodes at 1e-10."""
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    p, v = layered_nt6
    with WaveHoltz(p, precision="fp64") as wh:
        got = to_np(wh.apply_S(v))
        info = L.ewh_get_info(wh.ctx)
    assert info.nt == 6 and info.kernel_variant[0] < VARIANT_RESIDENT
    plan = [0, 8, 19, 132, 117, 54, 768, 5]  # any partition: only its node positions are used
    nodes, _ = _sample_nodes(plan, *p.n)
    gv = _gather(p, got, nodes)
    scale = np.abs(got).max()
    for nd, g in zip(nodes, gv):
        want = window_sample(p, info.nt, v, nd, reach=4)
        assert np.abs(g - want).max() <= 1e-10 * scale, (nd, g, want)


def test_resident_1024_whole_field_matches_split(layered_nt6, monkeypatch):
    """Every node of the 1024^2 resident S v (the benchmark's CTA shape)
    against the oracle-checked FP32 split kernels."""
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    p, v = layered_nt6
    monkeypatch.setenv("EWH_STEP2D_O4", "split")
    with WaveHoltz(p, precision="fp32") as wh:
        a = to_np(wh.apply_S(v))
        assert L.ewh_get_info(wh.ctx).kernel_variant[1] < VARIANT_RESIDENT
    monkeypatch.setenv("EWH_STEP2D_O4", "r1")
    with WaveHoltz(p, precision="fp32") as wh:
        b = to_np(wh.apply_S(v))
        assert L.ewh_get_info(wh.ctx).kernel_variant[1] == VARIANT_RESIDENT + 1
    assert rel_err(b, a) < 2 * tol32(6)


def test_grid_wait_gives_up_and_context_recovers(monkeypatch):
    """A zero grid-wait limit makes every barrier wait of the resident launch
    give up at once: S v comes back NaN and the give-up is counted; the FP32
    solve sees the breakdown and finishes on the FP64 operator (status 0, the
    oracle's residual); with the limit restored the same context returns
    the same S v as before."""
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    monkeypatch.setenv("EWH_STEP2D_O4", "r0")
    p = inputs.small_problem(2, [40, 34], 4, [D, D, D, F, 0, 0], seed=42)  # M(I - S) definite
    s = O.build_system(p)
    v = inputs.random_vectors(p, 1, 61)[0]
    with WaveHoltz(p, precision="fp32") as wh:
        good = to_np(wh.apply_S(v))
        assert L.ewh_get_info(wh.ctx).kernel_variant[1] == VARIANT_RESIDENT
        assert rel_err(good, O.apply_S(s, v)) < tol32(s.nt)
        with pytest.raises(L.EwhError):
            wh.set_grid_wait(-1)
        wh.reset_stats()
        wh.set_grid_wait(0)
        bad = to_np(wh.apply_S(v))
        assert np.isnan(bad).all()
        assert wh.stats().grid_wait_timeouts == 1
        x, info = wh.solve(tol=1e-8)
        assert info.status == 0 and info.rel_res <= 1e-8
        assert wh.stats().grid_wait_timeouts >= 2
        x = to_np(x)
        b = O.apply_Pi0(s)
        r = b - (x - O.apply_S(s, x))
        assert math.sqrt(O.mdot(s, r, r) / O.mdot(s, b, b)) <= 1.01e-8
        wh.set_grid_wait(10 ** 9)
        again = to_np(wh.apply_S(v))
        assert np.array_equal(again, good)
        assert wh.stats().grid_wait_timeouts >= 2
