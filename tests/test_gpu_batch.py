"""Batches (row a7): several independent problems of different sizes,
frequencies and right-hand-side counts advanced together.  Every member's S
apply and solve must equal the same problem solved alone (identical kernels in
the same order: bitwise in FP64) and the oracle."""
import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs
from _helpers import TOL64, oracle_all_rhs, rel_err, to_np, tol32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _members(order):
    # three sizes, three frequencies, 1-3 shots each
    out = []
    for k, (nu, scale, nrhs) in enumerate([(40, 1.0, 2), (56, 0.75, 1), (72, 0.5, 3)]):
        L = (nu + 1) * 0.01
        shots = [L * (j + 1) / (nrhs + 1) for j in range(nrhs)]
        out.append(inputs.cfg_layered_2d(nu=nu, order=order, nrhs=nrhs, shot_x=shots, ppw=12.0,
                                         omega_scale=scale))
    return out


@pytest.mark.parametrize("order", [2, 4])
def test_batch_apply_S_matches_single_and_oracle(order):
    from paper_2205_12344_gb300.api import WaveHoltz, WaveHoltzBatch
    probs = _members(order)
    vs = [inputs.random_vectors(p, 1, 50 + k)[0] for k, p in enumerate(probs)]
    with WaveHoltzBatch(probs, "fp64") as wb:
        outs = [to_np(o) for o in wb.apply_S(vs)]
    for p, v, o in zip(probs, vs, outs):
        with WaveHoltz(p) as wh:
            single = to_np(wh.apply_S(v))
        assert np.array_equal(o, single)
        s = O.build_system(p)
        assert rel_err(o, oracle_all_rhs(s, lambda ss, x, r: O.apply_S(ss, x, r), v)) < TOL64


def test_batch_solve_fp64_equals_single_solves():
    from paper_2205_12344_gb300.api import WaveHoltz, WaveHoltzBatch
    probs = _members(4)
    with WaveHoltzBatch(probs, "fp64") as wb:
        xs, infos = wb.solve(tol=1e-9, maxit=5000)
    for p, x, inf in zip(probs, xs, infos):
        with WaveHoltz(p) as wh:
            xs1, inf1 = wh.solve(tol=1e-9, maxit=5000)
        assert inf.status == 0 and inf1.status == 0
        assert inf.iters == inf1.iters
        assert np.array_equal(to_np(x), to_np(xs1))
        s = O.build_system(p)
        n = s.K.shape[0]
        for r in range(p.nrhs):
            v = O.helmholtz_direct(s, r)
            assert np.linalg.norm(to_np(x)[r * n:(r + 1) * n] - v) <= 1e-6 * np.linalg.norm(v)


def test_batch_solve_fp32_reaches_fp64_residual():
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    probs = _members(4)
    with WaveHoltzBatch(probs, "fp32") as wb:
        xs, infos = wb.solve(tol=1e-7, maxit=20000)
        launches = wb.kernel_launches()
    for p, x, inf in zip(probs, xs, infos):
        assert inf.status == 0
        assert inf.rel_res <= 1e-7
        s = O.build_system(p)
        n = s.K.shape[0]
        for r in range(p.nrhs):
            v = O.helmholtz_direct(s, r)
            assert np.linalg.norm(to_np(x)[r * n:(r + 1) * n] - v) <= 1e-4 * np.linalg.norm(v)
    assert launches > 0
