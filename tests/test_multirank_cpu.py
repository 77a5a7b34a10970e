"""The multi-rank layout (independent systems per rank) on CPU gloo ranks:
round-robin sharding, max-time / total-work reduction and result gathering
reproduce a single-process run of the same systems (solved here by the FP64
oracle, which stands in for the per-GPU solver on CPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2205_12344_gb300 import parallel


def test_shard_partitions_items():
    for n in (0, 1, 5, 192):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in parallel.shard(n, r, world))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        parallel.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import ewh_oracle as O
    from paper_2205_12344_gb300 import inputs
    n_items = 5
    mine = parallel.shard(n_items, rank, world)
    local = []
    for i in mine:
        p = inputs.small_problem(2, [7, 6], 2, [0, 0, 0, 1], seed=i)
        s = O.build_system(p)
        local.append(O.apply_Pi0(s).tolist())
    t, w = parallel.reduce_job(0.5 + rank, len(mine))
    allres = parallel.gather_results(local, n_items, rank, world)
    q.put((rank, t, w, allres))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_serial():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import ewh_oracle as O
    from paper_2205_12344_gb300 import inputs
    serial = []
    for i in range(5):
        s = O.build_system(inputs.small_problem(2, [7, 6], 2, [0, 0, 0, 1], seed=i))
        serial.append(O.apply_Pi0(s))
    for rank, t, w, allres in outs:
        assert t == 1.5            # slowest rank
        assert w == 5              # every item counted once
        for a, b in zip(allres, serial):
            assert np.array_equal(np.asarray(a), b)
