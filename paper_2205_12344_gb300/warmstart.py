"""Learned warm start for the El-WaveHoltz solve (the warm-start form).

A 4-level convolutional encoder-decoder with skip connections (channels
32/64/128/128, 3x3 convolutions, leaky ReLU, 2x2 average pooling, nearest
upsampling) maps per-node features of the medium, the forcing and the
frequency -- and the method's own first two vectors, the right-hand side
b = Pi 0 and S b (eq. amat_sym), which carry the phase of the wave field --
to a guess y of the solution's shape.  Weights and activations are BF16,
accumulation FP32; every layer (forward, backward, Adam) runs in libewh.so's
kernels; PyTorch only provides device memory and the stream.

Use: x0 = c1 y + c2 b with (c1, c2) minimising ||b - A x0||_M (A = I - S;
A b = b - S b is known, A y costs one S apply), which never raises the
initial residual above ||b||_M: the plain solve stays the fallback, and the
solve's stopping rule (the FP64 residual) decides the result whatever the
start.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib as L

IN_CH = 16     # input features, zero-padded to the 16-channel granule
OUT_CH = 16    # head width (the first two channels are the guess)


def features(prob, b=None, sb=None):
    """Per-unknown-node input features [H, W, IN_CH] (FP32) of a 2D problem
    with Dirichlet sides: log Vs, log(Vp/Vs), log rho, normalised forcing,
    frequency relative to the 10-points-per-wavelength frequency, the node
    coordinates and, when given, b = Pi 0 and S b (solver layout, scaled by
    the RMS of b)."""
    assert prob.dim == 2 and all(b == 0 for b in prob.bc[:4]), "warm start: 2D, Dirichlet sides"
    sl = (slice(1, -1), slice(1, -1))
    rho, lam, mu = prob.rho[sl], prob.lam[sl], prob.mu[sl]
    vs = np.sqrt(mu / rho)
    vp = np.sqrt((lam + 2 * mu) / rho)
    f = prob.forcing[0][:, 1:-1, 1:-1]
    fmax = max(np.abs(f).max(), 1e-30)
    H, W = vs.shape
    h = prob.h
    w10 = 2 * math.pi * vs.min() / (10 * h)
    ys, xs = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, W), indexing="ij")
    out = np.zeros((H, W, IN_CH), dtype=np.float32)
    out[..., 0] = np.log(vs) / 0.2
    out[..., 1] = np.log(vp / vs) - math.log(1.8)
    out[..., 2] = np.log(rho)
    out[..., 3] = f[0] / fmax
    out[..., 4] = f[1] / fmax
    out[..., 5] = prob.omega / w10 - 0.75
    out[..., 6] = xs
    out[..., 7] = ys
    if b is not None:
        bb = np.asarray(b, dtype=np.float64).reshape(2, H, W)
        rms = math.sqrt(float(np.mean(bb ** 2))) or 1.0
        out[..., 8] = bb[0] / rms
        out[..., 9] = bb[1] / rms
        if sb is not None:
            s2 = np.asarray(sb, dtype=np.float64).reshape(2, H, W)
            out[..., 10] = s2[0] / rms
            out[..., 11] = s2[1] / rms
    return out


def target(prob, v):
    """Solution [2 * H * W] (unknown nodes) -> [H, W, 2] normalised to unit RMS."""
    H, W = prob.n[1] - 2, prob.n[0] - 2
    t = np.asarray(v, dtype=np.float64).reshape(2, H, W).transpose(1, 2, 0)
    rms = math.sqrt(float(np.mean(t ** 2))) or 1.0
    return (t / rms).astype(np.float32)


class WarmStartNet:
    """The encoder-decoder; parameters live on the GPU (FP32 master + BF16 copy)."""

    def __init__(self, H, W, channels=(32, 64, 128, 128), seed=0):
        import torch
        assert H % 8 == 0 and W % 8 == 0, "three poolings need H, W divisible by 8"
        self.torch = torch
        self.H, self.W = H, W
        c1, c2, c3, c4 = channels
        self.c = channels
        # (name, Ci, Co, leaky, level) ; level = resolution divisor exponent
        self.spec = [("e1a", IN_CH, c1, 1, 0), ("e1b", c1, c1, 1, 0),
                     ("e2a", c1, c2, 1, 1), ("e2b", c2, c2, 1, 1),
                     ("e3a", c2, c3, 1, 2), ("e3b", c3, c3, 1, 2),
                     ("m_a", c3, c4, 1, 3), ("m_b", c4, c4, 1, 3),
                     ("d3a", c4 + c3, c3, 1, 2), ("d3b", c3, c3, 1, 2),
                     ("d2a", c3 + c2, c2, 1, 1), ("d2b", c2, c2, 1, 1),
                     ("d1a", c2 + c1, c1, 1, 0), ("d1b", c1, c1, 1, 0),
                     ("head", c1, OUT_CH, 0, 0)]
        rng = np.random.default_rng(seed)
        dev = "cuda"
        self.params = {}
        for name, ci, co, act, _ in self.spec:
            std = math.sqrt(2.0 / (9 * ci)) * (0.1 if name == "head" else 1.0)
            w = torch.tensor(rng.standard_normal((co, 3, 3, ci)) * std, dtype=torch.float32, device=dev)
            b = torch.zeros(co, dtype=torch.float32, device=dev)
            self.params[name] = {"w": w, "b": b, "w_bf": w.to(torch.bfloat16).contiguous(),
                                 "mw": torch.zeros_like(w), "vw": torch.zeros_like(w),
                                 "mb": torch.zeros_like(b), "vb": torch.zeros_like(b),
                                 "gw": torch.zeros_like(w), "gb": torch.zeros_like(b)}
        self.step_count = 0
        self.scratch = torch.empty(9 * 256 * 256, dtype=torch.bfloat16, device=dev)

    # -- helpers
    def _empty(self, shape, dtype):
        return self.torch.empty(shape, dtype=dtype, device="cuda")

    def _conv(self, name, x, N, h, w, st):
        _, ci, co, act, _ = next(s for s in self.spec if s[0] == name)
        p = self.params[name]
        pre = self._empty((N, h, w, co), self.torch.float32)
        out = self._empty((N, h, w, co), self.torch.bfloat16)
        L.ewh_conv3x3_fwd(x, p["w_bf"], p["b"], pre, out, act, N, h, w, ci, co, st)
        return pre, out

    def forward(self, x, stream=None):
        """x: BF16 [N, H, W, IN_CH] -> FP32 [N, H, W, OUT_CH]; keeps what backward needs."""
        t = self.torch
        N = x.shape[0]
        H, W = self.H, self.W
        c1, c2, c3, c4 = self.c
        st = stream
        cache = {"x": x, "N": N}
        dims = [(H >> k, W >> k) for k in range(4)]

        def conv(name, inp, lvl):
            h, w = dims[lvl]
            pre, out = self._conv(name, inp, N, h, w, st)
            cache[name] = (inp, pre, out)
            return out

        def pool(a, lvl, c):
            h, w = dims[lvl]
            out = self._empty((N, h // 2, w // 2, c), t.bfloat16)
            L.ewh_avgpool2(a, out, N, h, w, c, st)
            return out

        def up_cat(low, lvl_low, c_low, skip, c_skip):
            h, w = dims[lvl_low]
            cat = self._empty((N, 2 * h, 2 * w, c_low + c_skip), t.bfloat16)
            L.ewh_upsample2(low, cat, N, h, w, c_low, c_low + c_skip, 0, st)
            L.ewh_copy_channels(skip, cat, N * 4 * h * w, c_skip, c_low + c_skip, c_low, st)
            return cat

        s1 = conv("e1b", conv("e1a", x, 0), 0)
        s2 = conv("e2b", conv("e2a", pool(s1, 0, c1), 1), 1)
        s3 = conv("e3b", conv("e3a", pool(s2, 1, c2), 2), 2)
        m = conv("m_b", conv("m_a", pool(s3, 2, c3), 3), 3)
        d3 = conv("d3b", conv("d3a", up_cat(m, 3, c4, s3, c3), 2), 2)
        d2 = conv("d2b", conv("d2a", up_cat(d3, 2, c3, s2, c2), 1), 1)
        d1 = conv("d1b", conv("d1a", up_cat(d2, 1, c2, s1, c1), 0), 0)
        _, pre, _ = cache["head"] = (d1,) + self._conv("head", d1, N, H, W, st)
        self.cache = cache
        return pre

    def backward(self, dout, stream=None):
        """dout: FP32 [N, H, W, OUT_CH] = d(loss)/d(output); fills every
        parameter's gradient (gw, gb)."""
        t = self.torch
        c = self.cache
        N = c["N"]
        H, W = self.H, self.W
        c1, c2, c3, c4 = self.c
        st = stream
        dims = [(H >> k, W >> k) for k in range(4)]

        def conv_back(name, d_out, lvl):
            """d_out: FP32 gradient w.r.t. the layer's output (activation);
            returns the FP32 gradient w.r.t. its input."""
            _, ci, co, act, _ = next(s for s in self.spec if s[0] == name)
            h, w = dims[lvl]
            inp, pre, _ = c[name]
            p = self.params[name]
            n = N * h * w * co
            g = self._empty((N, h, w, co), t.float32)
            g_bf = self._empty((N, h, w, co), t.bfloat16)
            if act:
                L.ewh_leaky_relu_bwd(pre, d_out, g, g_bf, n, st)
            else:
                g = d_out
                L.ewh_f32_to_bf16(g, g_bf, n, st)
            L.ewh_bias_grad(g, p["gb"], N * h * w, co, st)
            L.ewh_conv3x3_wgrad(inp, g_bf, p["gw"], N, h, w, ci, co, st)
            dx = self._empty((N, h, w, ci), t.float32)
            L.ewh_conv3x3_dgrad(g_bf, p["w_bf"], self.scratch, dx, N, h, w, ci, co, st)
            return dx

        def split_up_cat(d_cat, lvl_low, c_low, c_skip, d_skip):
            """gradient of up_cat: returns d(low) and accumulates into d_skip."""
            h, w = dims[lvl_low]
            d_low = self._empty((N, h, w, c_low), t.float32)
            L.ewh_upsample2_bwd(d_cat, d_low, N, h, w, c_low, c_low + c_skip, 0, st)
            L.ewh_slice_channels(d_cat, d_skip, N * 4 * h * w, c_skip, c_low + c_skip, c_low, 1, st)
            return d_low

        def pool_back(d_pooled, lvl, ch, into):
            h, w = dims[lvl]
            g = self._empty((N, h, w, ch), t.float32)
            L.ewh_avgpool2_bwd(d_pooled, g, N, h, w, ch, st)
            L.ewh_slice_channels(g, into, N * h * w, ch, ch, 0, 1, st)     # into += g

        d1 = conv_back("head", dout, 0)
        d_s1 = t.zeros((N, H, W, c1), dtype=t.float32, device="cuda")
        d_s2 = t.zeros((N, H // 2, W // 2, c2), dtype=t.float32, device="cuda")
        d_s3 = t.zeros((N, H // 4, W // 4, c3), dtype=t.float32, device="cuda")
        d_cat1 = conv_back("d1a", conv_back("d1b", d1, 0), 0)
        d_d2 = split_up_cat(d_cat1, 1, c2, c1, d_s1)
        d_cat2 = conv_back("d2a", conv_back("d2b", d_d2, 1), 1)
        d_d3 = split_up_cat(d_cat2, 2, c3, c2, d_s2)
        d_cat3 = conv_back("d3a", conv_back("d3b", d_d3, 2), 2)
        d_m = split_up_cat(d_cat3, 3, c4, c3, d_s3)
        d_p3 = conv_back("m_a", conv_back("m_b", d_m, 3), 3)
        pool_back(d_p3, 2, c3, d_s3)
        d_p2 = conv_back("e3a", conv_back("e3b", d_s3, 2), 2)
        pool_back(d_p2, 1, c2, d_s2)
        d_p1 = conv_back("e2a", conv_back("e2b", d_s2, 1), 1)
        pool_back(d_p1, 0, c1, d_s1)
        conv_back("e1a", conv_back("e1b", d_s1, 0), 0)

    def adam(self, lr=1e-3, stream=None):
        self.step_count += 1
        for p in self.params.values():
            L.ewh_adam_step(p["w"], p["gw"], p["mw"], p["vw"], p["w_bf"], p["w"].numel(), lr, 0.9, 0.999, 1e-8,
                            self.step_count, stream)
            L.ewh_adam_step(p["b"], p["gb"], p["mb"], p["vb"], None, p["b"].numel(), lr, 0.9, 0.999, 1e-8,
                            self.step_count, stream)

    def loss_and_grad(self, y, tgt, stream=None):
        """Mean over the batch of 1/2 ||y - t||^2 / ||t||^2 on the two solution
        channels; returns (per-sample losses, FP32 gradient)."""
        t = self.torch
        N = y.shape[0]
        P = self.H * self.W
        grad = self._empty(tuple(y.shape), t.float32)
        loss = self._empty((N,), t.float32)
        L.ewh_scaled_l2_loss(y, tgt, grad, loss, P, OUT_CH, 2, N, stream)
        return loss, grad


def guess_to_vector(y_hw2):
    """[H, W, 2] guess -> solver layout [2 * H * W] (FP64 numpy)."""
    a = np.asarray(y_hw2, dtype=np.float64)
    return np.ascontiguousarray(a.transpose(2, 0, 1)).reshape(-1)


# ---------------------------------------------------------------------------
# Data, training and the with/without comparison
# ---------------------------------------------------------------------------

def make_media(count, nu, seed0, order=2, ppw=None):
    """GRF media (log Vs std 0.2, correlation 0.1, Vp = 1.8 Vs, rho = 1) on the
    unit square with nu^2 unknowns, a Gaussian source (sigma 2h) at a random
    interior position, and a frequency uniform in [0.5, 1] x the
    10-points-per-wavelength frequency, or (ppw = (lo, hi)) giving a number of
    points per shortest wavelength uniform in [lo, hi]."""
    from . import inputs
    rng = np.random.default_rng(seed0)
    probs = []
    for k in range(count):
        if ppw is None:
            kw = {"omega_scale": float(rng.uniform(0.5, 1.0))}
        else:
            kw = {"ppw": float(rng.uniform(ppw[0], ppw[1]))}
        src = (float(rng.uniform(0.2, 0.8)), float(rng.uniform(0.2, 0.8)))
        probs.append(inputs.cfg_grf_2d(nu=nu, order=order, seed=seed0 + k, src=src, **kw))
    return probs


def solve_all(probs, tol, chunk=16, precision="fp32", log=None):
    """Solutions with the batched solver (FP64 residual <= tol), and each
    problem's b = Pi 0 and S b (the network's phase inputs)."""
    from .api import WaveHoltzBatch
    sols, bs, sbs = [], [], []
    for i in range(0, len(probs), chunk):
        if log:
            log("solutions %d / %d" % (i, len(probs)))
        with WaveHoltzBatch(probs[i:i + chunk], precision) as wb:
            b = wb.apply_Pi0()
            sb = wb.apply_S(b)
            xs, infos = wb.solve(tol=tol, maxit=200000, raise_on_error=False)
            sols += [x.cpu().numpy() for x in xs]
            bs += [x.cpu().numpy() for x in b]
            sbs += [x.cpu().numpy() for x in sb]
    return sols, bs, sbs


def train(net, feats, targets, epochs, batch, lr=1e-3, seed=0, log=None):
    """Minibatch Adam on the scaled L2 loss; returns the per-epoch mean loss."""
    import torch
    rng = np.random.default_rng(seed)
    X = torch.tensor(np.stack(feats), dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    T = torch.tensor(np.stack(targets), dtype=torch.float32).cuda().contiguous()
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for i in range(0, n - batch + 1, batch):
            idx = torch.tensor(order[i:i + batch], device="cuda")
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            y = net.forward(xb)
            loss, grad = net.loss_and_grad(y, tb)
            net.backward(grad)
            net.adam(lr)
            tot += float(loss.sum())
        hist.append(tot / (n - n % batch))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return hist


def predict(net, feat):
    import torch
    x = torch.tensor(feat[None], dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    return net.forward(x)[0, :, :, :2].cpu().numpy()


def warm_start_vector(wh, y_hw2, b=None, sb=None):
    """x0 = c1 y + c2 b, (c1, c2) minimising ||b - A x0||_M over the span of
    the guess and b (A = I - S with the context's S apply, its working
    precision; A b = b - S b): the residual of x0 is never larger than that of
    the zero start, nor than that of the best multiple of b.  Without b, the
    best multiple of y.  Returns (x0, (c1, c2))."""
    y = guess_to_vector(y_hw2)
    yt = wh._vec(y)
    Ay = yt - wh.apply_S(yt)
    if b is None:
        b = wh.apply_Pi0()
        num = wh.mdot(b, Ay)[0]
        den = wh.mdot(Ay, Ay)[0]
        alpha = num / den if den > 0 else 0.0
        return yt * alpha, (alpha, 0.0)
    b = wh._vec(b)
    Ab = b - (wh._vec(sb) if sb is not None else wh.apply_S(b))
    g11, g12, g22 = wh.mdot(Ay, Ay)[0], wh.mdot(Ay, Ab)[0], wh.mdot(Ab, Ab)[0]
    r1, r2 = wh.mdot(Ay, b)[0], wh.mdot(Ab, b)[0]
    det = g11 * g22 - g12 * g12
    if det > 1e-14 * g11 * g22:
        c1 = (r1 * g22 - r2 * g12) / det
        c2 = (r2 * g11 - r1 * g12) / det
    else:  # y (nearly) parallel to b: the best multiple of b
        c1, c2 = 0.0, (r2 / g22 if g22 > 0 else 0.0)
    return yt * c1 + b * c2, (c1, c2)


def compare(net, probs, tol, precision="fp32"):
    """Iterations and time to tol with and without the warm start (the
    warm-start time includes inference and the scaling apply)."""
    import time
    import torch
    from .api import WaveHoltz
    rows = []
    for p in probs:
        with WaveHoltz(p, precision=precision) as wh:
            wh.solve(tol=tol, maxit=200000, raise_on_error=False)      # warm graphs
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, i0 = wh.solve(tol=tol, maxit=200000, raise_on_error=False)
            torch.cuda.synchronize()
            t_plain = time.perf_counter() - t0
            t0 = time.perf_counter()
            b = wh.apply_Pi0()
            sb = wh.apply_S(b)
            y = predict(net, features(p, b.cpu().numpy(), sb.cpu().numpy()))
            x0, coef = warm_start_vector(wh, y, b, sb)
            xw, iw = wh.solve(tol=tol, maxit=200000, x0=x0, raise_on_error=False)
            torch.cuda.synchronize()
            t_warm = time.perf_counter() - t0
            r0 = b - (x0 - wh.apply_S(x0))
            bb = wh.mdot(b, b)[0]
            rel0 = math.sqrt(wh.mdot(r0, r0)[0] / bb)
            # the method without the network: the best multiple of b
            Ab = b - sb
            cb = wh.mdot(Ab, b)[0] / wh.mdot(Ab, Ab)[0]
            rb = b - Ab * cb
            relb = math.sqrt(wh.mdot(rb, rb)[0] / bb)
        rows.append({"iters_plain": i0.iters, "iters_warm": iw.iters, "t_plain": t_plain, "t_warm": t_warm,
                     "rel_res_x0": rel0, "rel_res_b": relb, "coef": coef, "status": (i0.status, iw.status)})
    return rows


def run_experiment(n_train=512, n_test=32, nu=256, epochs=30, batch=8, tol=1e-6, seed=0, log=None, order=2,
                   ppw=None, lr=1e-3, train_tol=None):
    """Generate solutions (to train_tol, default tol), train the network on
    the GPU, compare solves to tol with and without the warm start."""
    import time
    t0 = time.perf_counter()
    probs = make_media(n_train + n_test, nu, seed, order=order, ppw=ppw)
    sols, bs, sbs = solve_all(probs[:n_train], train_tol or tol, log=log)
    t_gen = time.perf_counter() - t0
    feats = [features(p, b, sb) for p, b, sb in zip(probs[:n_train], bs, sbs)]
    targs = [target(p, v) for p, v in zip(probs[:n_train], sols)]
    net = WarmStartNet(nu, nu, seed=seed)
    t0 = time.perf_counter()
    hist = train(net, feats, targs, epochs, batch, lr=lr, log=log)
    t_train = time.perf_counter() - t0
    rows = compare(net, probs[n_train:], tol)
    ip = [r["iters_plain"] for r in rows]
    iw = [r["iters_warm"] for r in rows]
    tp = [r["t_plain"] for r in rows]
    tw = [r["t_warm"] for r in rows]
    return {"n_train": n_train, "n_test": n_test, "nu": nu, "epochs": epochs, "tol": tol, "order": order,
            "train_tol": train_tol or tol,
            "ppw": ppw, "rel_res_b_mean": float(np.mean([r["rel_res_b"] for r in rows])),
            "seconds_generate": t_gen, "seconds_train": t_train, "loss_first": hist[0], "loss_last": hist[-1],
            "iters_plain_mean": float(np.mean(ip)), "iters_warm_mean": float(np.mean(iw)),
            "iters_plain_median": float(np.median(ip)), "iters_warm_median": float(np.median(iw)),
            "time_plain_mean": float(np.mean(tp)), "time_warm_mean": float(np.mean(tw)),
            "rel_res_x0_mean": float(np.mean([r["rel_res_x0"] for r in rows])),
            "rows": rows}


def main(argv=None):
    """The warm-start experiment from the command line; writes the result as JSON."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-test", type=int, default=200)
    ap.add_argument("--nu", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--ppw", type=float, nargs=2, default=None, help="points per wavelength range")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--train-tol", type=float, default=None, help="residual of the training solutions (default: tol)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None, help="JSON file for the result")
    a = ap.parse_args(argv)
    import sys
    res = run_experiment(n_train=a.n_train, n_test=a.n_test, nu=a.nu, epochs=a.epochs, batch=a.batch, tol=a.tol,
                         seed=a.seed, order=a.order, ppw=tuple(a.ppw) if a.ppw else None, lr=a.lr,
                         train_tol=a.train_tol,
                         log=lambda m: print(m, file=sys.stderr, flush=True))
    text = json.dumps(res, indent=1, default=float)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    summary = {k: v for k, v in res.items() if k != "rows"}
    print(json.dumps(summary, default=float))


if __name__ == "__main__":
    main()
