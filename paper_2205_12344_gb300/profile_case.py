"""A small, self-contained run of the step kernels for profilers (ncu).

Applies S (one period of the corrected leapfrog with the trapezoid filter,
eqs. (qoper) and (elastic-time-explicit-corrected)) a few times to a random
vector on the layered 2D medium of the benchmark (order-4 SBP operator,
1024^2 nodes by default), then exits.  Every launch it makes is one of the
library's own kernels; the state is ~60 MB per right-hand side in FP32, so a
capture of one or two launches stays small.

    python -m paper_2205_12344_gb300.profile_case --nu 1024 --nrhs 1 --precision fp32 --applies 2

With ``--mapping annulus`` the same medium sits on a curvilinear grid: the
(q, r) square mapped onto an annular sector of about the same extent (the
mapped-grid step kernels of Section 4.1).  With ``--grf3d`` the workload is
the 3D Gaussian-random-field cube instead (``--nu`` nodes per axis, order 4).
The step kernel is the autotuner's choice unless EWH_STEP2D_O4 /
EWH_STEP3D_O4 name one.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nu", type=int, default=1024, help="nodes per axis")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides (shots) per launch")
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp64"))
    ap.add_argument("--applies", type=int, default=2, help="applications of S")
    ap.add_argument("--mapping", default="none", choices=("none", "annulus"), help="curvilinear grid")
    ap.add_argument("--grf3d", action="store_true", help="3D random-field cube instead of the layered 2D medium")
    a = ap.parse_args(argv)

    import torch

    from . import inputs
    from .api import WaveHoltz

    if a.grf3d:
        p = inputs.cfg_grf_3d(nu=a.nu, order=4)
    else:
        p = inputs.cfg_layered_2d(nu=a.nu, order=4, nrhs=a.nrhs, shot_x=[2.0 + 1.5 * k for k in range(a.nrhs)])
    if a.mapping == "annulus" and not a.grf3d:
        L = (p.n[0] - 1) * p.h
        p.mapping = inputs.annulus_mapping(p.n, p.h, span=0.5, r0=1.5 * L, dr=L)
    with WaveHoltz(p, precision=a.precision) as wh:
        g = torch.Generator(device="cuda").manual_seed(7)
        v = torch.randn(wh.n, dtype=torch.float64, device="cuda", generator=g)
        o = None
        for _ in range(a.applies):
            o = wh.apply_S(v)
        torch.cuda.synchronize()
        info = wh.stats()
        k = 0 if a.precision == "fp64" else 1
        print("applies %d  |S v| %.6e  launches %d  nt %d  ms/level %.4f" %
              (a.applies, float(o.norm()), int(info.launches), int(wh.info.nt),
               info.wave_ms[k] / max(info.steps[k], 1)))


if __name__ == "__main__":
    main()
