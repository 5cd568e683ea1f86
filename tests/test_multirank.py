"""The multi-process path of bench.py on CPU: two `gloo` ranks on 127.0.0.1.

Every rank solves its own replica over disjoint sample ids (weak scaling, no
data-path collective); the job's time is the slowest rank's.  Each rank samples
its ids with the oracle; rank 0 checks that the ranks' sets are exactly the
slices of one single-process run over all ids and that the timing reduction
returns the maximum.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, theta, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_2408_10982_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = inputs.rmat_graph(1 << 11, 1 << 15, 3, "lt")
        first = bench.replica_first_id(rank, theta)
        pool = O.sample(O.LT, g, 42, first, theta)
        sizes = [None] * world
        dist.all_gather_object(sizes, (rank, first, pool.set_off.tolist(), pool.members.tolist()))
        slowest = bench.max_over_ranks(float(10 + rank), dist)
        if rank == 0:
            out.put((sizes, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_replicas():
    pytest.importorskip("torch")
    import multiprocessing as mp
    import oracle as O
    from paper_2408_10982_gb300 import inputs
    world, theta = 2, 500
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, theta, out)) for r in range(world)]
    for p in procs:
        p.start()
    got, slowest = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert slowest == 10.0 + (world - 1)
    g = inputs.rmat_graph(1 << 11, 1 << 15, 3, "lt")
    whole = O.sample(O.LT, g, 42, 0, world * theta)
    for rank, first, set_off, members in sorted(got):
        assert first == rank * theta
        lo, hi = whole.set_off[first], whole.set_off[first + theta]
        assert np.array_equal(np.asarray(members, np.int32), whole.members[lo:hi])
        assert np.array_equal(np.asarray(set_off, np.int64), whole.set_off[first:first + theta + 1] - lo)
