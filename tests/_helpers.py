"""Shared helpers for the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on identical seeded inputs)."""
import numpy as np

from oracle import ewh_oracle as O
from paper_2205_12344_gb300 import inputs

# FP64 GPU vs oracle (the stated bar): relative l2 and max-norm error.
TOL64 = 1e-10
# FP32 stencil vs FP64 oracle for one S or Pi apply.  Rounding of the FP32
# state (unit roundoff 2^-24 = 6e-8) accumulates over the N leapfrog levels
# and the N+1 filter terms roughly like a random walk, with an O(1) factor
# from the stencil's cancellation at 10 points per wavelength:
#     err <~ C sqrt(N) 2^-24,  C = 30  ->  2e-6 at N = 120, 3e-6 at N = 265.
def tol32(nsteps):
    return 30.0 * np.sqrt(nsteps) * 2.0 ** -24


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    d = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    m = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    return max(d, m)


def oracle_all_rhs(s, fn, vecs):
    """Apply an oracle function per right-hand side to stacked vectors."""
    n = s.K.shape[0]
    out = []
    for r in range(len(vecs) // n):
        out.append(fn(s, vecs[r * n:(r + 1) * n], r))
    return np.concatenate(out)


def to_np(t):
    return t.detach().cpu().numpy()


def window_sample(prob, nt, v, node_xyz, reach):
    """Oracle S v at one node via its domain of dependence: crop the problem to
    a window of radius (N+2)*reach nodes around the node (held at zero
    outside; N = nt * periods leapfrog levels, ``reach`` = stencil radius) and
    apply S there.  Returns the dim components of (S v) at the node."""
    N = nt * prob.periods
    R = (N + 2) * reach
    dim = prob.dim
    lo = [max(0, node_xyz[a] - R) for a in range(dim)]
    hi = [min(prob.n[a] - 1, node_xyz[a] + R) for a in range(dim)]
    w = inputs.window_problem(prob, lo, hi)
    sw = O.build_system(w, nt=nt)
    idx = inputs.unknown_index(prob)
    widx = inputs.unknown_index(w)
    nn, wnn = prob.n_nodes(), w.n_nodes()
    sl = tuple(slice(lo[a], hi[a] + 1) for a in reversed(range(dim)))
    sub = idx[sl]
    ok = widx >= 0
    vw = np.zeros(dim * wnn)
    for c in range(dim):
        vw[c * wnn + widx[ok]] = v[c * nn + sub[ok]]
    outw = O.apply_S(sw, vw)
    loc = tuple(node_xyz[a] - lo[a] for a in reversed(range(dim)))
    return np.array([outw[c * wnn + widx[loc]] for c in range(dim)])
