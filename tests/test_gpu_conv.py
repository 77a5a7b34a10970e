"""Warm-start layer kernels (BF16 tensor-core convolutions with FP32
accumulation and the element-wise layers) against the FP64 layer oracle on the
same BF16-rounded inputs: only the FP32 accumulation order differs."""
import numpy as np
import pytest

from oracle import conv_oracle as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_12344_gb300 import build
    build.build()


def _bf(a):
    """FP64 array -> (CUDA bf16 tensor, the same values back in FP64)."""
    t = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    return t, t.float().cpu().double().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("N,H,W,Ci,Co,act", [(1, 8, 8, 16, 8, 0), (2, 13, 70, 32, 48, 1), (1, 32, 64, 96, 32, 1),
                                             (2, 16, 16, 16, 128, 0)])
def test_conv_forward(N, H, W, Ci, Co, act):
    from paper_2205_12344_gb300 import _lib as L
    rng = np.random.default_rng(N * 1000 + Ci + Co)
    xt, x = _bf(rng.standard_normal((N, H, W, Ci)))
    wt, w = _bf(rng.standard_normal((Co, 3, 3, Ci)) / np.sqrt(9 * Ci))
    b = rng.standard_normal(Co)
    bt = torch.tensor(b, dtype=torch.float32).cuda()
    pre = torch.empty((N, H, W, Co), dtype=torch.float32, device="cuda")
    actt = torch.empty((N, H, W, Co), dtype=torch.bfloat16, device="cuda")
    L.ewh_conv3x3_fwd(xt, wt, bt, pre, actt, act, N, H, W, Ci, Co)
    torch.cuda.synchronize()
    ref = C.conv3x3(x, w, b.astype(np.float32).astype(np.float64))
    assert _rel(pre.cpu().double().numpy(), ref) < 2e-5
    ref_act = C.leaky_relu(ref) if act else ref
    assert _rel(actt.float().cpu().double().numpy(), ref_act) < 1e-2   # bf16 output rounding


@pytest.mark.parametrize("N,H,W,Ci,Co", [(1, 8, 8, 16, 16), (2, 12, 40, 32, 64), (1, 16, 64, 96, 32)])
def test_conv_gradients(N, H, W, Ci, Co):
    from paper_2205_12344_gb300 import _lib as L
    rng = np.random.default_rng(7 + Ci + Co)
    xt, x = _bf(rng.standard_normal((N, H, W, Ci)))
    wt, w = _bf(rng.standard_normal((Co, 3, 3, Ci)) / np.sqrt(9 * Ci))
    dyt, dy = _bf(rng.standard_normal((N, H, W, Co)))
    dx = torch.empty((N, H, W, Ci), dtype=torch.float32, device="cuda")
    scratch = torch.empty(9 * Ci * Co, dtype=torch.bfloat16, device="cuda")
    L.ewh_conv3x3_dgrad(dyt, wt, scratch, dx, N, H, W, Ci, Co)
    dw = torch.empty((Co, 3, 3, Ci), dtype=torch.float32, device="cuda")
    L.ewh_conv3x3_wgrad(xt, dyt, dw, N, H, W, Ci, Co)
    torch.cuda.synchronize()
    assert _rel(dx.cpu().double().numpy(), C.conv3x3_dgrad(dy, w)) < 2e-5
    assert _rel(dw.cpu().double().numpy(), C.conv3x3_wgrad(x, dy)) < 1e-4


def test_elementwise_layers():
    from paper_2205_12344_gb300 import _lib as L
    rng = np.random.default_rng(3)
    N, H, W, Cc = 2, 8, 12, 16
    xt, x = _bf(rng.standard_normal((N, H, W, Cc)))
    y = torch.empty((N, H // 2, W // 2, Cc), dtype=torch.bfloat16, device="cuda")
    L.ewh_avgpool2(xt, y, N, H, W, Cc)
    up = torch.zeros((N, H, W, 48), dtype=torch.bfloat16, device="cuda")
    L.ewh_upsample2(y, up, N, H // 2, W // 2, Cc, 48, 16)
    cat = torch.zeros((N, H, W, 48), dtype=torch.bfloat16, device="cuda")
    L.ewh_copy_channels(xt, cat, N * H * W, Cc, 48, 32)
    dyt = torch.tensor(rng.standard_normal((N, H, W, 48)), dtype=torch.float32).cuda()
    g_up = torch.empty((N, H // 2, W // 2, Cc), dtype=torch.float32, device="cuda")
    L.ewh_upsample2_bwd(dyt, g_up, N, H // 2, W // 2, Cc, 48, 16)
    g_pool = torch.empty((N, H, W, Cc), dtype=torch.float32, device="cuda")
    L.ewh_avgpool2_bwd(g_up, g_pool, N, H, W, Cc)
    sl = torch.full((N, H, W, Cc), 1.0, dtype=torch.float32, device="cuda")
    L.ewh_slice_channels(dyt, sl, N * H * W, Cc, 48, 32, 1)
    db = torch.empty(48, dtype=torch.float32, device="cuda")
    L.ewh_bias_grad(dyt, db, N * H * W, 48)
    pre = torch.tensor(rng.standard_normal((N, H, W, Cc)), dtype=torch.float32).cuda()
    gl = torch.empty_like(pre)
    L.ewh_leaky_relu_bwd(pre, g_pool, gl, None, pre.numel())
    torch.cuda.synchronize()
    pooled = C.avgpool2(x)
    assert _rel(y.float().cpu().double().numpy(), pooled) < 1e-2
    yb = y.float().cpu().double().numpy()
    assert np.array_equal(up.float().cpu().double().numpy()[..., 16:32], C.upsample2(yb))
    assert np.array_equal(cat.float().cpu().double().numpy()[..., 32:48], x)
    dyn = dyt.cpu().double().numpy()
    gu = C.upsample2_grad(dyn[..., 16:32])
    assert _rel(g_up.cpu().double().numpy(), gu) < 1e-6
    assert _rel(g_pool.cpu().double().numpy(), C.avgpool2_grad(gu)) < 1e-6
    assert _rel(sl.cpu().double().numpy(), 1.0 + dyn[..., 32:48]) < 1e-6
    assert _rel(db.cpu().double().numpy(), C.bias_grad(dyn)) < 1e-5
    assert _rel(gl.cpu().double().numpy(), C.leaky_relu_grad(pre.cpu().double().numpy(),
                                                              C.avgpool2_grad(gu))) < 1e-6


def test_adam_matches_its_definition():
    """Adam (Kingma and Ba 2015): m, v moving averages, bias correction."""
    from paper_2205_12344_gb300 import _lib as L
    rng = np.random.default_rng(4)
    n = 1000
    p0 = rng.standard_normal(n)
    p = torch.tensor(p0, dtype=torch.float32).cuda()
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    pr, mr, vr = p0.copy(), np.zeros(n), np.zeros(n)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    for step in range(1, 6):
        g = rng.standard_normal(n)
        L.ewh_adam_step(p, torch.tensor(g, dtype=torch.float32).cuda(), m, v, pb, n, lr, b1, b2, eps, step)
        mr = b1 * mr + (1 - b1) * g
        vr = b2 * vr + (1 - b2) * g * g
        pr = pr - lr * (mr / (1 - b1 ** step)) / (np.sqrt(vr / (1 - b2 ** step)) + eps)
    torch.cuda.synchronize()
    assert _rel(p.cpu().double().numpy(), pr) < 1e-5
    assert _rel(pb.float().cpu().double().numpy(), pr) < 1e-2
