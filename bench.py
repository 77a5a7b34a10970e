#!/usr/bin/env python
"""Benchmark of the El-WaveHoltz hot path on GB300.

Workload: the 2D layered seismic medium (1024 x 1024 unknowns + free top row,
h = 10 m, 8 layers, Vp 1.5-4.5 km/s, Vs = Vp/sqrt(3), rho 1.8-2.6 g/cc,
traction-free top, Dirichlet elsewhere, w for 10 points per shear wavelength,
Ricker source), fourth-order SBP stencil, FP32 stencil with FP64 Krylov.

One step = one pass of the whole hot path from a cold start: Pi 0 (forced FP64
wave solve), then ITERS iterations of CG in the M inner product on the FP32
operator (each one FP32 S apply = nt leapfrog levels with the trapezoid
filter, plus the FP64 Krylov updates), FP64 true-residual replacements, and
the final FP64 residual.  A complete solve of this workload to 1e-6 needs
tens of thousands of iterations (cond(I - S) ~ w^(2d)), far beyond a bench
step, so the time-to-1e-6 comparison against the plain FP64 GPU solve is
measured on smaller layered media of the same family (and on the 64 x 64
homogeneous case), solved to tolerance by both.

value = grid-point updates (nodes x leapfrog levels over every wave solve of
the step, FP32 and FP64) per second, whole job.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; every rank solves its own shot
(weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpt-updates/s, HBM % of peak; time to 1e-6 residual vs plain FP64 GPU solve"
UNIT = "Gpt-updates/s"
ALG_BYTES_2D_FP32 = 52.0      # bytes per grid-point update of one unfused leapfrog+filter pass
# floating-point operations per node-level of the order-4 step kernels' interior
# path (FMA = 2), counted from the kernels: 2D 29 (stresses) + 37 (divergence and
# update); 3D 61 + 73
FLOPS_PER_NODE_LEVEL = {2: 66.0, 3: 134.0}
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nu", type=int, default=1024)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--iters", type=int, default=100, help="CG iterations per step")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 GPU solve used for the time-to-tol comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 192-system measurement")
    ap.add_argument("--batch-full-tol", action="store_true",
                    help="also extrapolate the full 192-system batch's time to 1e-6 from measured per-member "
                         "solves (minutes of GPU time; off by default)")
    ap.add_argument("--batch-iters", type=int, default=100, help="batched CG iterations timed")
    ap.add_argument("--no-device-loop", action="store_true",
                    help="skip the timing of the step with CG windows under device control")
    ap.add_argument("--no-mapped", action="store_true", help="skip the mapped-grid (annular sector) measurement")
    ap.add_argument("--mapped-applies", type=int, default=4, help="S applies timed per precision on the mapped grid")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D order-4 measurement")
    ap.add_argument("--nu3d", type=int, default=256, help="unknowns per axis of the 3D workload")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(nu, rank, world):
    from paper_2205_12344_gb300 import inputs, parallel
    # each rank solves its own shot (independent problems, weak scaling)
    L = (nu + 1) * 0.01
    shot = parallel.shot_positions(L, world)[parallel.shard(world, rank, world)[0]]
    return inputs.cfg_layered_2d(nu=nu, order=4, shot_x=[shot])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ewh_stencil.cu", "ewh_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2205_12344_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def step_kernel_name(variant):
    """The 2D order-4 FP32 step kernel behind an autotuner variant number."""
    tiles = {0: "32x8", 1: "32x16", 2: "64x8", 3: "64x4"}
    shapes = {5: "1024, 4", 6: "768, 5", 7: "512, 7"}
    if variant in tiles:
        return "sbp_stress2d_tl + sbp_div2d_tl (%s tiles), per time level" % tiles[variant]
    if variant == 4:
        return "step2d_o4_fused, per time level"
    if variant in shapes:
        return "step2d_o4_resident<%s> (all levels of a wave solve in one cooperative launch), per time level" % shapes[variant]
    return "unknown variant %d" % variant


def fma_peaks():
    """Measured FMA throughput of this GPU (TFLOP/s, FP64 and FP32) from the
    library's probe kernel."""
    from paper_2205_12344_gb300 import _lib as L
    return {"fp64": L.ewh_fma_rate(L.EWH_FP64) / 1e12, "fp32": L.ewh_fma_rate(L.EWH_FP32_STENCIL) / 1e12}


def alu_roofline(flops_per_node_level, nodes, step_ms, peak_tflops, what):
    """Arithmetic roofline of a step kernel: its interior operation count per
    node-level x nodes / the measured per-level time, against the measured
    FMA rate of its precision."""
    achieved = flops_per_node_level * nodes / (step_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "flops_per_node_level": flops_per_node_level,
            "peak_source": "measured (ewh_fma_rate)", "kernel": what}


def traffic_per_step(nodes):
    """DRAM bytes per leapfrog step of the dominant kernels from the committed
    ncu summary, scaled to ``nodes``; None when absent or stale."""
    p = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_node_step"]) * nodes


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(prob, nt, window_nodes=512, min_seconds=8.0):
    """Time the FP64 oracle's S apply on a bounded window of the workload
    (domain-of-dependence crop; single host thread).  Returns (Gpt/s, desc)."""
    import numpy as np
    from oracle import ewh_oracle as O
    from paper_2205_12344_gb300 import inputs
    cx = prob.n[0] // 2
    half = window_nodes // 2
    lo = [cx - half, prob.n[1] - window_nodes]
    hi = [cx + half - 1, prob.n[1] - 1]
    w = inputs.window_problem(prob, lo, hi)
    s = O.build_system(w, nt=nt)
    v = np.random.default_rng(0).standard_normal(s.K.shape[0])
    reps = 0
    t0 = time.perf_counter()
    while True:
        O.apply_S(s, v)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    upd = reps * w.n_nodes() * nt
    return upd / el / 1e9, {"window": "%dx%d nodes by the free top" % (window_nodes, window_nodes),
                            "s_applies": reps, "seconds": round(el, 2)}


_POOL_SYSTEM = {}


def _oracle_pool_init(nu, nt, window_nodes, kind="layered2d"):
    """Build, once per host process, the oracle system of a window of the
    layered 2D workload (by the free top) or of the 3D random-field cube (at
    its centre); S applies only: the source plays no part."""
    import numpy as np
    from oracle import ewh_oracle as O
    from paper_2205_12344_gb300 import inputs
    half = window_nodes // 2
    if kind == "grf3d":
        prob = inputs.cfg_grf_3d(nu=nu, order=4)
        c = prob.n[0] // 2
        w = inputs.window_problem(prob, [c - half] * 3, [c + half - 1] * 3)
    else:
        prob = inputs.cfg_layered_2d(nu=nu, order=4)
        cx = prob.n[0] // 2
        w = inputs.window_problem(prob, [cx - half, prob.n[1] - window_nodes], [cx + half - 1, prob.n[1] - 1])
    _POOL_SYSTEM["s"] = O.build_system(w, nt=nt)
    _POOL_SYSTEM["v"] = np.random.default_rng(os.getpid()).standard_normal(_POOL_SYSTEM["s"].K.shape[0])
    _POOL_SYSTEM["updates"] = w.n_nodes() * nt


def _oracle_pool_run(args):
    """S applies from ``start_at`` until ``seconds`` have passed: (updates,
    start, end) in wall-clock seconds."""
    seconds, start_at = args
    from oracle import ewh_oracle as O
    while time.time() < start_at:
        time.sleep(0.005)
    reps, t0 = 0, time.time()
    while True:
        O.apply_S(_POOL_SYSTEM["s"], _POOL_SYSTEM["v"])
        reps += 1
        if time.time() - t0 >= seconds:
            break
    return reps * _POOL_SYSTEM["updates"], t0, time.time()


class OraclePool:
    """The FP64 oracle on every host core: one spawned process per core
    (numpy and scipy single-threaded in each), each holding the same window
    of the layered workload.  ``round(seconds)`` runs S applies on all of
    them at once and returns the aggregate grid-point updates per second
    (total updates over the span from the first start to the last end)."""

    ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __init__(self, nu, nt, window_nodes, workers=None, kind="layered2d"):
        import multiprocessing as mp
        self.workers = workers or len(os.sched_getaffinity(0))
        self.window_nodes = window_nodes
        self.kind = kind
        saved = {k: os.environ.get(k) for k in self.ENV}
        for k in self.ENV:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers, _oracle_pool_init, (nu, nt, window_nodes, kind))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def round(self, seconds):
        start_at = time.time() + 0.2
        # the first map also waits for every process to build its window
        res = self.pool.map(_oracle_pool_run, [(seconds, start_at)] * self.workers, chunksize=1)
        upd = sum(r[0] for r in res)
        span = max(r[2] for r in res) - min(r[1] for r in res)
        return upd / span / 1e9, span

    def describe(self, span):
        if self.kind == "grf3d":
            where = "a %d^3-node window at the centre of the cube" % self.window_nodes
        else:
            where = "a %dx%d-node window by the free top" % (self.window_nodes, self.window_nodes)
        return ("oracle FP64 S apply on %d host processes at once (one core each), each on %s, %.1f s" %
                (self.workers, where, span))

    def close(self):
        self.pool.close()
        self.pool.join()


def time_to_tol_table(flush, stream):
    """Time to a relative FP64 residual of 1e-6 (1e-8 for the homogeneous case)
    for the plain FP64 GPU solve and the FP32-stencil / FP64-Krylov solve, each
    timed with CUDA events after one untimed warm solve."""
    import torch
    from paper_2205_12344_gb300 import inputs
    from paper_2205_12344_gb300.api import WaveHoltz
    cases = [("homogeneous2d_64 (64x64, order 2, w=10)", inputs.cfg_homogeneous_2d(nu=64, omega=10.0), 1e-8),
             ("layered2d_256 (256x256 + free top, order 4, 10 PPW)", inputs.cfg_layered_2d(nu=256, order=4), 1e-6)]
    out = []
    for name, prob, tol in cases:
        row = {"workload": name, "tol": tol}
        sols = {}
        for prec in ("fp64", "fp32"):
            wh = WaveHoltz(prob, precision=prec)
            wh.solve(tol=tol, maxit=200000, raise_on_error=False)
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = wh.solve(tol=tol, maxit=200000, raise_on_error=False)
            e1.record(stream)
            e1.synchronize()
            sols[prec] = x
            row[prec] = {"seconds": e0.elapsed_time(e1) / 1e3, "iters": info.iters, "rel_res": info.rel_res,
                         "status": info.status, "s_applies_fp32": info.s_applies,
                         "s_applies_fp64": info.s_applies_fp64}
            wh.close()
        row["speedup_mixed_vs_fp64"] = row["fp64"]["seconds"] / row["fp32"]["seconds"]
        row["solution_rel_diff"] = float(torch.linalg.norm(sols["fp32"] - sols["fp64"]) /
                                         torch.linalg.norm(sols["fp64"]))
        out.append(row)
    return out


def batch_members(nu_list=(256, 384, 512), scales=(0.5, 0.75, 1.0), shots=64):
    """64 shots x 3 frequencies on layered media of 256^2, 384^2 and 512^2
    unknowns (h = 10 m, same layered profile): shot i sits on size i mod 3, at
    evenly spaced surface positions; one member per (size, frequency) carrying
    its size's shots as right-hand sides (192 systems in 9 members)."""
    from paper_2205_12344_gb300 import inputs, parallel
    members = []
    for si, nu in enumerate(nu_list):
        nshots = len(range(si, shots, len(nu_list)))
        xs = parallel.shot_positions((nu + 1) * 0.01, nshots)
        for sc in scales:
            members.append(inputs.cfg_layered_2d(nu=nu, order=4, nrhs=nshots, shot_x=xs, omega_scale=sc))
    return members


def batch_measurement(iters, stream):
    """Throughput of the batched mixed-precision solve: Pi 0 setup of every
    member plus ``iters`` batched CG iterations (every member advances one
    FP32 S apply per iteration), timed with CUDA events."""
    import torch
    from paper_2205_12344_gb300.api import WaveHoltzBatch
    members = batch_members()
    systems = sum(p.nrhs for p in members)
    with WaveHoltzBatch(members, "fp32") as wb:
        wb.solve(tol=1e-6, maxit=2, raise_on_error=False)          # warm: graphs, autotuner
        torch.cuda.synchronize()
        l0 = wb.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs, infos = wb.solve(tol=1e-6, maxit=iters, raise_on_error=False)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        launches = wb.kernel_launches() - l0
        levels = 0
        for p, inf, info in zip(members, infos, wb.infos):
            levels += (inf.s_applies + inf.s_applies_fp64) * info.nt * p.nrhs * info.nodes
    return {"workload": "64 shots x 3 frequencies (0.5, 0.75, 1.0 x w10) on layered 256^2/384^2/512^2, "
                        "order 4, FP32 stencil + FP64 CG, 9 members / 192 systems",
            "systems": systems, "iters": iters, "seconds": ms / 1e3,
            "value": levels / (ms * 1e-3) / 1e9, "unit": UNIT, "gpu_launches": launches,
            "max_rel_res": max(i.rel_res for i in infos)}


ALG_BYTES_MAPPED = {"fp32": 68.0, "fp64": 136.0}   # 52 (104) B plus the 4 metric planes per node


def mapped_workload(nu):
    """The benchmark's layered medium and source on a curvilinear grid: the
    (q, r) square mapped onto an annular sector of about the same extent
    (radius 1.5 L .. 2.5 L along q, 0.5 rad along r; L the side length)."""
    from paper_2205_12344_gb300 import inputs
    p = workload(nu, 0, 1)
    L = (p.n[0] - 1) * p.h
    p.mapping = inputs.annulus_mapping(p.n, p.h, span=0.5, r0=1.5 * L, dr=L)
    return p


def wave_measurement(prob, label, applies, alg_bytes, stream, flush, kernels):
    """S-apply throughput of one workload per precision: ``applies`` S applies
    (the first FP64 one only when ``applies[prec]`` is 1), the device time of
    the wave solves from the library's own CUDA events, the autotuner's kernel
    variant (named by ``kernels``) and a roofline against ``alg_bytes[prec]``
    per node-level."""
    import torch
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz
    out = {"workload": label}
    peak, peak_kind = peaks()
    for prec, idx in (("fp32", 1), ("fp64", 0)):
        if not applies.get(prec):
            continue
        with WaveHoltz(prob, precision=prec) as wh:
            g = torch.Generator(device="cuda").manual_seed(3)
            v = torch.randn(wh.n, dtype=torch.float64, device="cuda", generator=g)
            wh.apply_S(v)                                    # warm: autotuner, graph
            torch.cuda.synchronize()
            wh.reset_stats()
            ms = 0.0
            for _ in range(applies[prec]):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                wh.apply_S(v)
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
            st = wh.stats()
            nodes = int(wh.info.nodes)
            step_ms = st.wave_ms[idx] / max(st.steps[idx], 1)
            achieved = alg_bytes[prec] * nodes / (step_ms * 1e-3) / 1e9
            variant = int(L.ewh_get_info(wh.ctx).kernel_variant[idx])
            kname = kernels.get(variant, "variant %d" % variant)
            if prec == "fp64" and "fp64" in kernels:   # the fused FP32 kernels have no FP64 form
                kname = kernels["fp64"]
            out[prec] = {"value": st.steps[idx] * nodes / (ms * 1e-3) / 1e9, "unit": UNIT, "nt": int(wh.info.nt),
                         "nodes": nodes, "applies": applies[prec], "step_ms": step_ms,
                         "kernel": kname, "kernel_variant": variant,
                         "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                      "frac": achieved / peak, "peak_source": peak_kind,
                                      "alg_bytes_per_node_step": alg_bytes[prec]},
                         "gpu_launches": int(st.launches)}
    return out


def mapped_measurement(nu, applies, stream, flush):
    """Mapped-grid step (curvilinear order-4 SBP, Section 4.1) on the layered
    workload mapped onto an annular sector."""
    return wave_measurement(mapped_workload(nu),
                            "layered2d_%d on an annular sector (mapped grid), order-4 SBP, S applies" % nu,
                            {"fp32": applies, "fp64": applies}, ALG_BYTES_MAPPED, stream, flush,
                            {0: "curv_step2d (fused, 32x8)", 1: "curv_stress2d + curv_div2d",
                             2: "curv_step2d (fused, 32x16)"})


ALG_BYTES_3D = {"fp32": 72.0, "fp64": 144.0}      # read u, u_prev, acc + write u', acc (3 comps) + lambda, mu, 1/M


KERNELS_3D = {0: "sbp_stress + sbp_divergence_step (3D, per level)",
              1: "step3d_o4_zm<16> (fused z-march, 32x16 tiles, per level)",
              2: "step3d_o4_zm<8> (fused z-march, 32x8 tiles, per level)",
              "fp64": "sbp_stress + sbp_divergence_step (3D, per level; FP64 has no fused z-march)"}


def threed_measurement(nu, stream, flush, peaks_fma=None, small_nu=48, e2e_iters=5):
    """3D order-4 SBP step on the 256^3 Gaussian-random-field workload (log Vs
    GRF, Vp = 1.8 Vs, Dirichlet, point source at the centre): S-apply
    throughput per precision with its roofline (HBM; FP64 also against the
    measured FP64 FMA rate), the seconds per CG iteration, the end-to-end
    rate through the C ABI from host buffers, the oracle on every host core,
    and time to a 1e-6 residual on a reduced cube of the same family."""
    import numpy as np
    import torch
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300 import inputs
    from paper_2205_12344_gb300.api import WaveHoltz, make_desc
    prob = inputs.cfg_grf_3d(nu=nu, order=4)
    out = wave_measurement(prob, "grf3d_%d: 3D GRF medium %d^3 unknowns, order-4 SBP, S applies" % (nu, nu),
                           {"fp32": 2, "fp64": 1}, ALG_BYTES_3D, stream, flush, KERNELS_3D)
    nodes = out["fp32"]["nodes"]
    nt = out["fp32"]["nt"]
    for prec in ("fp32", "fp64"):
        out[prec]["seconds_per_cg_iteration"] = out[prec]["step_ms"] * nt * 1e-3
    if peaks_fma:
        out["fp64"]["alu_roofline"] = alu_roofline(FLOPS_PER_NODE_LEVEL[3], nodes, out["fp64"]["step_ms"],
                                                   peaks_fma["fp64"], "FP64 3D per-level order-4 pair")
    # end to end through the C ABI: create from pinned host buffers, a fixed
    # number of FP32-stencil CG iterations, the solution read into host memory
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k), dtype=np.float64)).pin_memory()
           for k in ("rho", "lam", "mu", "forcing")}
    out_host = torch.empty(prob.nrhs * prob.n_unknowns(), dtype=torch.float64).pin_memory()
    ms, upd = [], 0
    for k in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = L.ewh_create(make_desc(prob.dim, prob.n, prob.h, prob.order, prob.bc, L.EWH_FP32_STENCIL, prob.cfl),
                           pin["rho"], pin["lam"], pin["mu"], prob.omega, pin["forcing"], prob.nrhs,
                           stream.cuda_stream)
        L.ewh_solve(ctx, 1e-6, e2e_iters, None, out_host, raise_on_error=False)
        sts = L.ewh_get_stats(ctx)
        L.ewh_destroy(ctx)
        t1 = time.perf_counter()
        if k > 0:
            ms.append((t1 - t0) * 1e3)
            upd += all_levels(sts) * nodes
    out["e2e"] = {"value": upd / (sum(ms) * 1e-3) / 1e9, "unit": UNIT,
                  "h2d_bytes_per_step": sum(int(pin[k].numel()) * 8 for k in pin),
                  "d2h_bytes_per_step": int(out_host.numel()) * 8, "ms_per_step": statistics.mean(ms),
                  "step": "create from host buffers + FP64 Pi 0 + %d FP32-stencil CG iterations + FP64 residual, "
                          "solution to host" % e2e_iters}
    # time to 1e-6 on a reduced cube (the 256^3 cube needs O(1e4) iterations)
    small = inputs.cfg_grf_3d(nu=small_nu, order=4)
    row = {"workload": "grf3d_%d (same family, %d^3 unknowns), order 4, tol 1e-6" % (small_nu, small_nu)}
    for prec in ("fp64", "fp32"):
        with WaveHoltz(small, precision=prec) as wh:
            wh.apply_S(torch.zeros(wh.n, dtype=torch.float64, device="cuda"))   # untimed: autotuner, graphs
            torch.cuda.synchronize()
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = wh.solve(tol=1e-6, maxit=20000, raise_on_error=False)
            e1.record(stream)
            e1.synchronize()
            row[prec] = {"seconds": e0.elapsed_time(e1) / 1e3, "iters": info.iters, "rel_res": info.rel_res,
                         "status": info.status}
    row["speedup_mixed_vs_fp64"] = row["fp64"]["seconds"] / row["fp32"]["seconds"]
    out["time_to_tol_reduced"] = row
    return out


def threed_cpu_baseline(nu, nt, window_nodes=32, seconds=8.0):
    """The oracle's 3D S apply on every host core (a window of the cube)."""
    pool = OraclePool(nu, nt, window_nodes, kind="grf3d")
    pool.round(0.5)
    val, span = pool.round(seconds)
    desc = pool.describe(span)
    pool.close()
    return {"value": val, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": desc}


def batch_full_time_to_tol(stream, batch, tol=1e-6):
    """Time to a relative FP64 residual of ``tol`` for the full 192-system
    batch, EXTRAPOLATED from measured pieces (the batched solve itself runs
    longer than 1000 s): per member, one representative shot (the middle one)
    solved alone with the FP32-stencil solve to ``tol`` gives the member's
    iteration count; the batched time is the sum over members of those
    iterations times the member's share (by node-levels) of the measured
    per-iteration time of the full batch (``batch``: the 100-iteration
    measurement); the sequential plain FP64 arm is the sum over members of
    shots x iterations x the FP64 time per iteration, measured on the same
    shot as the difference of a 40- and a 10-iteration solve.  The batch's
    per-iteration time includes its FP64 setup and replacements (an
    overestimate for the batched arm)."""
    import torch
    from paper_2205_12344_gb300 import inputs, parallel
    from paper_2205_12344_gb300.api import WaveHoltz
    members = batch_members()
    scales = (0.5, 0.75, 1.0)
    t_iter = batch["seconds"] / batch["iters"]
    rows, work = [], []

    def timed_solve(q, prec, maxit):
        with WaveHoltz(q, precision=prec) as wh:
            wh.solve(tol=tol, maxit=2, raise_on_error=False)   # warm: graphs, autotuner
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = wh.solve(tol=tol, maxit=maxit, raise_on_error=False)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3, info, int(wh.info.nt), int(wh.info.nodes)

    for m, p in enumerate(members):
        nu = p.n[0] - 2
        xs_pos = parallel.shot_positions((nu + 1) * 0.01, p.nrhs)
        q = inputs.cfg_layered_2d(nu=nu, order=4, nrhs=1, shot_x=[xs_pos[p.nrhs // 2]],
                                  omega_scale=scales[m % len(scales)])
        s32, i32, nt, nodes = timed_solve(q, "fp32", 30000)
        s64a, i64a, _, _ = timed_solve(q, "fp64", 10)     # the difference of two lengths: per iteration,
        s64b, i64b, _, _ = timed_solve(q, "fp64", 40)     # without the Pi 0 setup and the final residual
        rows.append({"member": m, "nu": nu, "omega_scale": scales[m % len(scales)], "shots": p.nrhs,
                     "iters_to_tol_one_shot": i32.iters, "status": i32.status, "fp32_seconds_one_shot": s32,
                     "fp64_seconds_per_iter": (s64b - s64a) / max(i64b.iters - i64a.iters, 1)})
        work.append(nodes * nt * p.nrhs)
    W = float(sum(work))
    ok = [k for k, r in enumerate(rows) if r["status"] == 0]   # members whose shot reached tol
    batched = sum(rows[k]["iters_to_tol_one_shot"] * t_iter * work[k] / W for k in ok)
    seq = sum(rows[k]["shots"] * rows[k]["iters_to_tol_one_shot"] * rows[k]["fp64_seconds_per_iter"] for k in ok)
    return {"workload": "64 shots x 3 frequencies on layered 256^2/384^2/512^2, order 4: 192 systems", "tol": tol,
            "extrapolated": True, "maxit_representative": 30000,
            "members_converged": len(ok), "systems_covered": sum(rows[k]["shots"] for k in ok),
            "members_not_converged": [{"member": r["member"], "status": r["status"],
                                       "iters": r["iters_to_tol_one_shot"]} for r in rows if r["status"] != 0],
            "how": "iterations per member from one measured FP32 solve of its middle shot; batched = sum of "
                   "iterations x the member's node-level share of the measured full-batch time per iteration; "
                   "sequential FP64 = sum of shots x iterations x measured FP64 time per iteration; both sums over "
                   "the members whose shot converged (CG breaks down or stalls on near-resonant members)",
            "batched_seconds_extrapolated": batched, "sequential_fp64_seconds_extrapolated": seq,
            "speedup_extrapolated": seq / batched, "batch_seconds_per_iteration_measured": t_iter,
            "members": rows}


def batch_time_to_tol(stream, flush, tol=1e-6):
    """Time to a relative FP64 residual of ``tol`` for a reduced batch (8
    shots x 2 frequencies, 0.5 and 1.0 x w10, on layered 128^2 and 192^2: 16
    systems in 4 members): the batched FP32-stencil / FP64-Krylov solve
    against the same 16 systems solved one after another by the plain FP64
    solve.  Contexts are created untimed; each timed region is the solves.
    Both arms' solutions are compared with an accurate one (batched FP64 CG to
    a residual of 1e-10, untimed): equal residual is not equal error when
    cond(I - S) is 1e5..1e6."""
    import torch
    from paper_2205_12344_gb300 import inputs, parallel
    from paper_2205_12344_gb300.api import WaveHoltz, WaveHoltzBatch
    nu_list, scales, shots = (128, 192), (0.5, 1.0), 8
    members = batch_members(nu_list=nu_list, scales=scales, shots=shots)
    out = {"workload": "8 shots x 2 frequencies (0.5, 1.0 x w10) on layered 128^2/192^2, order 4: 16 systems",
           "tol": tol}
    with WaveHoltzBatch(members, "fp32") as wb:
        wb.solve(tol=tol, maxit=2, raise_on_error=False)          # warm: graphs, autotuner
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs, infos = wb.solve(tol=tol, maxit=200000, raise_on_error=False)
        e1.record(stream)
        e1.synchronize()
        xb = [x.clone() for x in xs]
        out["batched"] = {"seconds": e0.elapsed_time(e1) / 1e3, "max_iters": max(i.iters for i in infos),
                          "max_rel_res": max(i.rel_res for i in infos), "status": max(i.status for i in infos)}
    with WaveHoltzBatch(members, "fp64") as wa:                 # accurate solutions, untimed
        xa, ia = wa.solve(tol=1e-10, maxit=400000, raise_on_error=False)
        xa = [x.clone() for x in xa]
        out["accurate"] = {"tol": 1e-10, "max_rel_res": max(i.rel_res for i in ia),
                           "max_iters": max(i.iters for i in ia)}
    err_b = []
    for m, p in enumerate(members):
        n1 = xb[m].numel() // p.nrhs
        for r in range(p.nrhs):
            a = xa[m][r * n1:(r + 1) * n1]
            err_b.append(float(torch.linalg.norm(xb[m][r * n1:(r + 1) * n1] - a) / torch.linalg.norm(a)))
    out["batched"]["max_rel_err_vs_accurate"] = max(err_b)
    seq_s, seq_it, diffs, err_s = 0.0, 0, [], []
    for m, p in enumerate(members):
        si = nu_list.index(p.n[0] - 2)
        xs_pos = parallel.shot_positions((p.n[0] - 1) * 0.01, p.nrhs)
        sc = scales[m % len(scales)]
        n1 = xb[m].numel() // p.nrhs
        for r in range(p.nrhs):
            q = inputs.cfg_layered_2d(nu=nu_list[si], order=4, nrhs=1, shot_x=[xs_pos[r]], omega_scale=sc)
            with WaveHoltz(q, precision="fp64") as wh:
                wh.apply_Pi0()                                   # untimed: autotuner, forced graph
                torch.cuda.synchronize()
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x, info = wh.solve(tol=tol, maxit=200000, raise_on_error=False)
                e1.record(stream)
                e1.synchronize()
                seq_s += e0.elapsed_time(e1) / 1e3
                seq_it = max(seq_it, info.iters)
                xr = xb[m][r * n1:(r + 1) * n1]
                diffs.append(float(torch.linalg.norm(xr - x) / torch.linalg.norm(x)))
                a = xa[m][r * n1:(r + 1) * n1]
                err_s.append(float(torch.linalg.norm(x - a) / torch.linalg.norm(a)))
    out["sequential_fp64"] = {"seconds": seq_s, "max_iters": seq_it, "max_rel_err_vs_accurate": max(err_s)}
    out["speedup_batched_vs_sequential_fp64"] = seq_s / out["batched"]["seconds"]
    out["max_solution_rel_diff"] = max(diffs)
    return out


def run_reference(args, ws, rank):
    """--impl reference: the FP64 CPU oracle as it stands, on host cores."""
    if rank != 0:
        return
    from paper_2205_12344_gb300 import inputs
    from oracle import ewh_oracle as O
    prob = workload(args.nu, 0, 1)
    dtc = O.cfl_dt(2, 4, prob.h, prob.cfl, prob.rho, prob.lam, prob.mu)
    nt = max(5, int(math.ceil(2 * math.pi / prob.omega / dtc)))
    pool = OraclePool(args.nu, nt, 256)
    for _ in range(args.warmup):
        pool.round(0.3)
    upd_s, spans = [], []
    for _ in range(args.steps):
        v, span = pool.round(2.0)
        upd_s.append(v * span)
        spans.append(span)
    pool.close()
    value = sum(upd_s) / sum(spans)
    ms = statistics.mean(spans) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "layered2d_%d order-4 S apply (oracle sample, all host cores)" % args.nu,
                       "nt": nt, "l2": "oracle runs on the host"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "sample": "S applies on a 256x256-node window of the workload (nt=%d levels) on "
                                       "%d host processes at once, %d rounds of about 2 s" %
                                       (nt, pool.workers, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def device_loop_step(wh, one_solve, steps, flush, stream, nodes, host_ms):
    """The bench step again with the library's default: windows of up to 32
    CG iterations in one graph launch (a while-conditional node whose control
    kernel takes the host loop's decisions), the host polling once per
    window.  Same iterates; timed with CUDA events per step."""
    import torch
    one_solve()
    torch.cuda.synchronize()
    wh.reset_stats()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = wh.stats()
    return {"ms_per_step": sum(ms) / len(ms), "value": all_levels(st) * nodes / (sum(ms) * 1e-3) / 1e9,
            "unit": UNIT, "host_polled_ms_per_step": sum(host_ms) / len(host_ms),
            "note": "CG windows of up to 32 iterations in one graph launch (while-conditional node, device-side "
                    "control kernel); the host polls once per window"}


def all_levels(st):
    """Leapfrog levels of a context's stats: event-timed wave solves plus
    those inside device-controlled CG windows."""
    return st.steps[0] + st.steps[1] + st.loop_steps[0] + st.loop_steps[1]


def main():
    args = parse()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    from paper_2205_12344_gb300 import build
    build.build()
    from paper_2205_12344_gb300 import _lib as L
    from paper_2205_12344_gb300.api import WaveHoltz

    prob = workload(args.nu, rank, ws)
    wh = WaveHoltz(prob, precision="fp32")
    nodes = int(wh.info.nodes)
    nt = int(wh.info.nt)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_solve():
        return wh.solve(tol=args.tol, maxit=args.iters, raise_on_error=False)

    # The timed step polls the host after every CG iteration (EWH_CG_POLL=1),
    # so that every S apply is bracketed by the library's CUDA events (the
    # roofline's per-level time); the same step with the default window of
    # iterations under device control is timed after it ("device_loop").
    os.environ["EWH_CG_POLL"] = "1"
    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    wh.reset_stats()
    clock = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clock:
        clock.start()
    step_ms = []
    infos = []
    for _ in range(args.steps):
        flush.fill_(1.0)                      # L2 flush between timed steps (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = one_solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    barrier()
    clocks = clock.stop() if clock else None
    st = wh.stats()
    total_ms = sum(step_ms)
    updates = all_levels(st) * nodes
    from paper_2205_12344_gb300 import parallel
    total_ms, updates = parallel.reduce_job(total_ms, updates, device="cuda")
    value = updates / (total_ms * 1e-3) / 1e9
    # dominant kernel: the FP32 leapfrog step, per time level (the autotuner's
    # variant: per-level stress + divergence launches, or the resident launch
    # that runs every level of a wave solve)
    step_dev_ms = st.wave_ms[1] / max(st.steps[1], 1)
    from paper_2205_12344_gb300 import _lib as L
    variant = int(L.ewh_get_info(wh.ctx).kernel_variant[1])
    peak, peak_kind = peaks()
    achieved = ALG_BYTES_2D_FP32 * nodes / (step_dev_ms * 1e-3) / 1e9
    traffic = traffic_per_step(nodes)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": step_kernel_name(variant), "kernel_variant": variant,
                "alg_bytes_per_node_step": ALG_BYTES_2D_FP32,
                "fp64_step_ms": (st.wave_ms[0] / st.steps[0]) if st.steps[0] else None}
    launches = int(st.launches)
    it = [i.iters for i in infos]
    peaks_fma = fma_peaks() if rank == 0 else None
    if peaks_fma and st.steps[0]:
        roofline["fp64_alu"] = alu_roofline(FLOPS_PER_NODE_LEVEL[2], nodes, st.wave_ms[0] / st.steps[0],
                                            peaks_fma["fp64"], "FP64 per-level order-4 kernels (Pi 0 and the "
                                            "residual replacements of the step)")

    extra = {}
    # the same step with CG windows under device control (the library's default)
    os.environ.pop("EWH_CG_POLL", None)
    if not args.no_device_loop:
        extra["device_loop"] = device_loop_step(wh, one_solve, args.steps, flush, stream, nodes, step_ms)
    if rank == 0:
        extra["iters_per_step"] = args.iters
        extra["rel_res_after_step"] = max(i.rel_res for i in infos)
        extra["s_applies_fp32_per_step"] = infos[-1].s_applies
        extra["s_applies_fp64_per_step"] = infos[-1].s_applies_fp64
        if not args.no_fp64_compare:
            extra["time_to_tol"] = time_to_tol_table(flush, stream)
        if not args.no_batch:
            flush.fill_(1.0)
            extra["batch"] = batch_measurement(args.batch_iters, stream)
            extra["batch"]["time_to_tol"] = batch_time_to_tol(stream, flush)
            if args.batch_full_tol:
                extra["batch"]["time_to_tol_full"] = batch_full_time_to_tol(stream, extra["batch"])
        if not args.no_mapped:
            extra["mapped"] = mapped_measurement(args.nu, args.mapped_applies, stream, flush)
        if not args.no_3d:
            extra["grf3d"] = threed_measurement(args.nu3d, stream, flush, peaks_fma)
    wh.close()

    # end to end through the C ABI with host buffers: create (H2D of medium and
    # forcing from pinned memory) + solve (D2H of the solution into host memory)
    e2e = None
    if rank == 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k), dtype=np.float64)).pin_memory()
               for k in ("rho", "lam", "mu", "forcing")}
        out_host = torch.empty(prob.nrhs * prob.n_unknowns(), dtype=torch.float64).pin_memory()
        desc_args = dict(dim=prob.dim, n=prob.n, h=prob.h, order=prob.order, bc=prob.bc,
                         precision=L.EWH_FP32_STENCIL, cfl=prob.cfl, periods=prob.periods,
                         corrected=prob.corrected)
        from paper_2205_12344_gb300.api import make_desc
        e2e_ms = []
        e2e_updates = 0
        for k in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = L.ewh_create(make_desc(**desc_args), pin["rho"], pin["lam"], pin["mu"], prob.omega,
                               pin["forcing"], prob.nrhs, stream.cuda_stream)
            info = L.ewh_solve(ctx, args.tol, args.iters, None, out_host, raise_on_error=False)
            sts = L.ewh_get_stats(ctx)
            L.ewh_destroy(ctx)
            t1 = time.perf_counter()
            if k > 0:
                e2e_ms.append((t1 - t0) * 1e3)
                e2e_updates += all_levels(sts) * nodes
        h2d = sum(int(pin[k].numel()) * 8 for k in pin)
        d2h = int(out_host.numel()) * 8
        e2e = {"value": e2e_updates / (sum(e2e_ms) * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": statistics.mean(e2e_ms)}

    if rank == 0:
        cpu_val, cpu_desc = cpu_oracle_sample(prob, nt) if ws == 1 else (None, None)
        cpu_all = None
        if ws == 1 and "grf3d" in extra:
            extra["grf3d"]["cpu_baseline"] = threed_cpu_baseline(args.nu3d, extra["grf3d"]["fp32"]["nt"])
        if ws == 1:
            pool = OraclePool(args.nu, nt, 512)
            pool.round(0.5)                               # warm: every process has built its window
            val, span = pool.round(8.0)
            cpu_all = (val, pool.workers, pool.describe(span))
            pool.close()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 stencil / f64 krylov", "data": "synthetic",
            "config": {"workload": "layered2d_%d: 2D layered medium %dx%d unknowns + free top row, order-4 SBP, "
                                   "FP32 stencil + FP64 CG, %d iterations per step" % (args.nu, args.nu, args.nu,
                                                                                      args.iters),
                       "nodes": nodes, "nt": nt, "omega": prob.omega, "tol": args.tol,
                       "parallelism": "independent shots per GPU" if ws > 1 else "single GPU",
                       "l2": "flushed (256 MiB write) between timed steps"},
            "roofline": roofline,
            "cpu_baseline": ({"value": cpu_all[0], "unit": UNIT, "cores": cpu_all[1], "kind": "oracle",
                              "sample": cpu_all[2],
                              "single_thread": {"value": cpu_val, "unit": UNIT, "cores": 1,
                                                "sample": "oracle FP64 S apply, %s, %d applies in %.1f s" %
                                                          (cpu_desc["window"], cpu_desc["s_applies"],
                                                           cpu_desc["seconds"])}}
                             if cpu_all is not None else None),
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fma_peaks_tflops": peaks_fma,
        }
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
