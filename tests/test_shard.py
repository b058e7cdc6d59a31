"""Sharding one query's chunks over ranks (paper_2102_10768_gb300.shard).

On the CPU: the greedy split is a partition of the chunk list and balanced
within one chunk's estimate; the u64 count reduction is exact over two gloo
ranks on 127.0.0.1, including sums past 2^63 and a saturating overflow; and
two gloo ranks that each count their share of the oracle's own Alg. 2
partition (chunks as allowed sets) reduce to the query's full count.
On the GPU (one device, the ranks run one after another): the library's
chunk lists split by the same rule and matched share by share add up to the
whole count and the oracle's.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2102_10768_gb300 import shard  # noqa: E402  (host logic; loads no library)


def test_assign_chunks_partitions_and_balances():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        for _ in range(20):
            w = rng.integers(0, 1 << 20, size=int(rng.integers(0, 300))).astype(np.uint64)
            parts = shard.assign_chunks(w, world)
            assert len(parts) == world
            allidx = np.concatenate(parts) if parts else np.zeros(0, np.int64)
            assert sorted(allidx.tolist()) == list(range(w.shape[0]))          # each chunk once
            loads = [float(w[p].astype(np.float64).sum()) for p in parts]
            if w.shape[0]:
                assert max(loads) <= w.astype(np.float64).sum() / world + float(w.max()) + 1e-6
            assert all(np.array_equal(a, b) for a, b in zip(parts, shard.assign_chunks(w, world)))


def test_assign_chunks_by_hand():
    # 7, 5, 4, 3, 1 over two ranks: 7 -> r0, 5 -> r1, 4 -> r1 (5 < 7), 3 -> r0, 1 -> r1 (9 < 10)
    parts = shard.assign_chunks([4, 7, 1, 5, 3], 2)
    assert parts[0].tolist() == [1, 4] and parts[1].tolist() == [0, 2, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2102_10768_gb300 import shard as sh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        res = {}
        big = np.uint64(1 << 63) + np.uint64(12345)
        mine = np.array([rank + 1, (1 << 40) * (rank + 1), big if rank == 0 else 7, big, 0], np.uint64)
        s, over = sh.allreduce_counts(mine, dist)
        res["sums"] = [int(x) for x in s]
        res["over"] = over.tolist()
        # the oracle's Alg. 2 partition of one query, split by the greedy rule:
        # each rank counts its chunks (as allowed sets) and the counts are reduced
        import oracle
        rng = np.random.default_rng(44)
        n = 80
        e = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.12], np.int32)
        lab = rng.integers(0, 2, size=n).astype(np.int32)
        ql = np.array([0, 1, 0, 1], np.int32)
        qe = np.array([[0, 1], [1, 2], [2, 3], [0, 2]], np.int32)
        o = oracle.Graph(n, e, lab)
        oc = oracle.Cst(o, ql, qe)
        _, wi, _, _ = oc.workload()
        chunks = oc.partition(max(1, wi // 40))
        parts = sh.assign_chunks([c[4] for c in chunks], world)
        local = sum(oracle.count(o, ql, qe, allow=oc.chunk_allow(*chunks[i][:4])) for i in parts[rank])
        tot, _ = sh.allreduce_counts([local], dist)
        res["sharded"] = int(tot[0])
        res["whole"] = oracle.count(o, ql, qe)
        res["nchunks"] = len(chunks)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_sharded_counts_reduce_exactly_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        res = got[r]
        big = (1 << 63) + 12345
        assert res["sums"][0] == 3
        assert res["sums"][1] == 3 * (1 << 40)
        assert res["sums"][2] == big + 7 and not res["over"][2]
        assert res["sums"][3] == (1 << 64) - 1 and res["over"][3]        # 2^64 + 24690 saturates
        assert res["sums"][4] == 0
        assert res["nchunks"] > 4
        assert res["sharded"] == res["whole"] > 0


@pytest.mark.gpu
def test_gpu_chunk_shares_add_up():
    import oracle
    import paper_2102_10768_gb300 as F
    import synth
    F.build()
    w = synth.er_workload()
    g, o = F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)
    wg = synth.WalkGraph(w.n, w.edges)
    qs = [wg.query(w.labels, k, kind, 78, 10 * k + j) for k in (4, 5, 6) for j, kind in enumerate(("induced", "sparse"))]
    wg.close()
    qs += w.queries
    compared = 0
    ch = None
    for q in qs:
        r0 = oracle.match(o, q.labels, q.edges, budget=20_000_000)
        assert r0["complete"]
        cst = F.Cst(g, q.labels, q.edges)
        ch = F.Chunks(cst, F.default_config(delta_w=max(1, cst.W // 64), max_chunks=512))
        whole = F.match(cst, ch)["count"]
        assert whole == r0["count"]
        for world in (2, 3):
            parts = shard.assign_chunks(ch.weights(), world)
            tot = 0
            for p in parts:
                sub = ch.select(p)
                assert sub.n == len(p)
                assert sub.copy() == [ch.copy()[i] for i in p.tolist()]
                tot += F.match(cst, sub)["count"]
                sub.close()
            assert tot == whole
        compared += ch.n > 1
    assert compared >= 4
    with pytest.raises(F.FastError):
        ch.select([ch.n])
