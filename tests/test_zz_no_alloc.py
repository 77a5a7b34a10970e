"""The allocation-free weighted inner product (ewh_mdot_noalloc) gives the same
sums as the context's M inner product (ewh_mdot), on two calls in a row.

It exists for callers that cannot allocate device memory (during graph
capture, under a fixed memory budget, or inside another framework's pool):
it takes no context and keeps its scratch in a fixed array inside the
library.  This file is collected last so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def test_noalloc_matches_context_mdot_twice():
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    p = inputs.small_problem(2, [37, 29], 4, [0, 0, 0, 1], seed=23, nrhs=3)
    s = O.build_system(p)
    nodes = p.n_nodes()
    # the mass weight of each unknown node (the same for every component)
    w = torch.tensor(s.Mdiag[:nodes], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    with WaveHoltz(p) as wh:
        for call in range(2):
            x, y = inputs.random_vectors(p, 2, 40 + call)
            xt = torch.tensor(x, device="cuda")
            yt = torch.tensor(y, device="cuda")
            want = wh.mdot(xt, yt)
            out = torch.full((p.nrhs,), float("nan"), dtype=torch.float64, device="cuda")
            L.ewh_mdot_noalloc(xt, yt, w, nodes, p.dim, p.nrhs, out, stream.cuda_stream)
            stream.synchronize()
            got = out.cpu().numpy()
            for r in range(p.nrhs):
                assert abs(got[r] - want[r]) <= 1e-12 * abs(want[r]) + 1e-14, (call, r, got[r], want[r])


def test_noalloc_large_vectors_use_the_block_cap():
    """Above 65536 entries per member the call runs its 64-block cap with a
    grid-stride loop (ewh_mdot uses more blocks): the sums agree to rounding,
    on two calls in a row."""
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    p = inputs.small_problem(2, [200, 200], 2, [0, 0, 0, 1], seed=24, nrhs=2)
    s = O.build_system(p)
    nodes = p.n_nodes()
    assert p.dim * nodes > 65536
    w = torch.tensor(s.Mdiag[:nodes], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    with WaveHoltz(p) as wh:
        for call in range(2):
            x, y = inputs.random_vectors(p, 2, 50 + call)
            xt = torch.tensor(x, device="cuda")
            yt = torch.tensor(y, device="cuda")
            want = wh.mdot(xt, yt)
            out = torch.full((p.nrhs,), float("nan"), dtype=torch.float64, device="cuda")
            L.ewh_mdot_noalloc(xt, yt, w, nodes, p.dim, p.nrhs, out, stream.cuda_stream)
            stream.synchronize()
            got = out.cpu().numpy()
            scale = float(torch.sqrt((w.repeat(p.dim * p.nrhs) * xt * xt).sum() *
                                     (w.repeat(p.dim * p.nrhs) * yt * yt).sum()))
            for r in range(p.nrhs):
                assert abs(got[r] - want[r]) <= 1e-12 * scale, (call, r, got[r], want[r])


def test_noalloc_rejects_oversized_batch():
    from paper_2205_12344_gb300 import _lib as L
    x = torch.zeros(130 * 4, dtype=torch.float64, device="cuda")
    w = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(130, dtype=torch.float64, device="cuda")
    with pytest.raises(L.EwhError) as e:
        L.ewh_mdot_noalloc(x, x, w, 4, 1, 130, out)
    assert e.value.status == L.EWH_EINVAL
    assert "128" in str(e.value)
