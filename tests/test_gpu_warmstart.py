"""The learned warm start end to end on a small configuration: solutions
generated by the solver itself, the network trained on the GPU by the
library's forward/backward kernels, and the with/without comparison on
held-out media.  The network's output has no exact pin: the FP64 residual of
the solve decides whether it is good enough (the least-squares start never
raises the initial residual)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def test_network_gradient_matches_finite_differences():
    """d(loss)/d(bias of the head and of the first layer) from the library's
    backward pass vs central differences of the library's forward pass."""
    from paper_2205_12344_gb300 import warmstart as WS
    net = WS.WarmStartNet(16, 16, channels=(16, 16, 32, 32), seed=3)
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.standard_normal((2, 16, 16, WS.IN_CH)), dtype=torch.float32).to(torch.bfloat16).cuda()
    t = torch.tensor(rng.standard_normal((2, 16, 16, 2)), dtype=torch.float32).cuda()

    def loss():
        y = net.forward(x)
        l, g = net.loss_and_grad(y, t)
        return float(l.sum().double()) / 2, g

    _, g = loss()
    net.backward(g)
    # the loss is exactly quadratic in the head bias (large step is exact);
    # the first layer's bias acts through leaky ReLUs (small step)
    for name, k, eps in (("head", 0, 0.5), ("head", 1, 0.5), ("e1a", 3, 0.05)):
        p = net.params[name]
        analytic = float(p["gb"][k])
        old = float(p["b"][k])
        p["b"][k] = old + eps
        lp, _ = loss()
        p["b"][k] = old - eps
        lm, _ = loss()
        p["b"][k] = old
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - analytic) <= 0.05 * abs(fd) + 2e-3, (name, k, fd, analytic)


def test_warm_start_trains_and_reports_its_gain(record_property):
    """Train on solver-generated solutions, then solve held-out media with and
    without the warm start.  What is guaranteed is checked (the loss falls,
    the scaled start has a smaller residual than the zero start, both solves
    reach the FP64 tolerance); the gain in iterations and time is measured and
    recorded, not assumed: on oscillatory solutions it can be nil."""
    from paper_2205_12344_gb300 import warmstart as WS
    res = WS.run_experiment(n_train=48, n_test=6, nu=32, epochs=12, batch=8, tol=1e-6, seed=5)
    assert res["loss_last"] < 0.8 * res["loss_first"]
    assert res["rel_res_x0_mean"] < 1.0
    # the least-squares start over (guess, b) is never worse than the best multiple of b
    assert all(r["rel_res_x0"] <= r["rel_res_b"] * 1.001 + 1e-5 for r in res["rows"])  # FP32 S rounding
    assert all(r["status"] == (0, 0) for r in res["rows"])
    for k in ("iters_plain_mean", "iters_warm_mean", "time_plain_mean", "time_warm_mean", "rel_res_x0_mean"):
        record_property(k, res[k])
    print("warm start: iterations %.1f -> %.1f, time %.3f s -> %.3f s, initial residual %.3f of the zero start"
          % (res["iters_plain_mean"], res["iters_warm_mean"], res["time_plain_mean"], res["time_warm_mean"],
             res["rel_res_x0_mean"]))
