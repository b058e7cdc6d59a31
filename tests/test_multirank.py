"""The multi-rank path of bench.py on CPU: ranks are replicas that each
match their own queries (no data-path collective), and the job's numbers
are all ranks' embeddings over the slowest rank's time.  World size 2 over
gloo on 127.0.0.1."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: time 1 + r seconds, 10 (r + 1) embeddings; e2e 2 + r s, 5 (r + 1)
        r = bench.reduce_over_ranks([1.0 + rank, 10 * (rank + 1), 2.0 + rank, 5 * (rank + 1)], dist, "cpu")
        out.put((rank, r))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max time, summed work: (2 s, 30 embeddings, 3 s, 15 embeddings) on every rank
    assert got[0] == got[1] == (2.0, 30.0, 3.0, 15.0)


def test_ranks_draw_their_own_queries():
    """Replicas: every rank draws its own query set (its own seed); rank 0's
    is the 1,000-query batch the parity tests check against the oracle."""
    import bench
    seeds = [bench.query_seed(r) for r in range(64)]
    assert len(set(seeds)) == 64
    assert seeds[0] == 3000
