"""One system split into slabs over CPU gloo ranks (world size 2 and 3): the
halo exchange, the level blocking between exchanges and the exactly rounded
distributed inner products reproduce the undivided oracle bit for bit -- the
S apply and Pi 0 (Section 3, eq. qoper; Section 4.3) and every CG iterate
(Section 4.5, eq. amat_sym).  The oracle's sparse operator, restricted to
each rank's extended slab, is the local stepper; the decomposition logic
under test is paper_2205_12344_gb300.parallel."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2205_12344_gb300 import parallel

D, F = 0, 1

CASES = [  # (dim, unknown-ish grid, order, sides, levels per exchange, w)
    (2, [30, 24], 2, [D, D, D, F], 2, 8.0),
    (2, [20, 40], 4, [F, D, D, F], 2, 8.0),
    (3, [8, 7, 15], 2, [D, F, D, D, F, D], 3, 8.0),
]


def test_slab_ranges_and_validation():
    for n in (3, 10, 41):
        for world in (1, 2, 3):
            r = parallel.slab_ranges(n, world)
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        parallel.slab_ranges(2, 3)
    with pytest.raises(ValueError):
        parallel.Slab(2, 10, 5, 3, 0, halo=4)   # slabs of 3 or 4 planes < halo


def test_exactly_rounded_partials():
    rng = np.random.default_rng(5)
    v = rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000)
    for k in (1, 3, 7):
        parts = [p for c in np.array_split(v, k) for p in parallel.exact_partials(c.tolist())]
        assert math.fsum(parts) == math.fsum(v.tolist())


def _system(case):
    from oracle import ewh_oracle as O
    from paper_2205_12344_gb300 import inputs
    dim, nu, order, bc, _, omega = case
    p = inputs.small_problem(dim, nu, order, bc, seed=90 + order, omega=omega)
    s = O.build_system(p)
    nu_ax = [p.n[a] - (bc[2 * a] == D) - (bc[2 * a + 1] == D) for a in range(dim)]
    plane_size = int(np.prod(nu_ax[:-1]))
    return p, s, nu_ax[-1], plane_size


def _reach(s, plane_size):
    """Reach of M^{-1} K in planes of the slowest axis (from its sparsity)."""
    K = s.K.tocoo()
    nn = s.Mdiag.size // s.dim
    return int(np.max(np.abs((K.row % nn) // plane_size - (K.col % nn) // plane_size)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, case, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2205_12344_gb300 import inputs
        p, s, n_planes, plane_size = _system(case)
        R = _reach(s, plane_size)
        slab = parallel.Slab(s.dim, n_planes, plane_size, world, rank, halo=case[4] * R)
        E = slab.ext_global()
        own = slab.own_global()
        K_loc = s.K[E][:, E]
        M_loc = s.Mdiag[E]
        minvK = lambda u: (K_loc @ u) / M_loc        # the oracle's M^{-1} K on the slab
        zero = np.zeros(E.size)
        wave = lambda u0_own, g: parallel.slab_wave_solve(slab, minvK, u0_own, g, s.nt, s.periods, s.kt,
                                                          s.weights, R)
        v = inputs.random_vectors(p, 1, 91)[0]
        Sv = wave(v[own], zero)
        Pi0 = wave(np.zeros(own.size), s.f_over_rho[0][E])
        x, hist = parallel.slab_cg(lambda x_own: wave(x_own, zero), Pi0, s.Mdiag[own], world, tol=1e-9,
                                   maxit=400)
        q.put((rank, own, Sv, Pi0, x, hist, R))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "d%d_o%d_%s" % (c[0], c[2], "x".join(map(str, c[1]))))
def test_slab_ranks_match_undivided_oracle_bitwise(case, world):
    import multiprocessing as mp
    from oracle import ewh_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    outs = [q.get(timeout=600) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p, s, n_planes, plane_size = _system(case)
    from paper_2205_12344_gb300 import inputs
    v = inputs.random_vectors(p, 1, 91)[0]
    want_S = O.apply_S(s, v)
    want_P = O.apply_Pi0(s)
    xo, io = O.cg_solve(s, tol=1e-9, maxit=400)
    assert io.converged
    got_S, got_P, got_x = (np.full(want_S.size, np.nan) for _ in range(3))
    for rank, own, Sv, Pi0, x, hist, R in outs:
        got_S[own], got_P[own], got_x[own] = Sv, Pi0, x
        assert hist == io.history                     # every CG residual, bit for bit
        assert case[4] * R <= n_planes // world       # the halo really crosses ranks
    assert np.array_equal(got_S, want_S)
    assert np.array_equal(got_P, want_P)
    assert np.array_equal(got_x, xo)
