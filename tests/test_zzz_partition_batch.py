"""The batched partition (fast_partition_batch) against the per-query one.

Each CST's chunk list from one batched call must equal, element by element
and in order, what fast_partition gives for it with the same configuration
(which the oracle's Alg. 2 pins elsewhere): over several delta_w, with the
max_chunks cap hit or not, with sampling, with CSTs of no embedding, and
with a NULL CST reported per entry.  Matching over the batched chunks gives
the same counts.
"""

import numpy as np
import pytest

import paper_2102_10768_gb300 as F
import synth

pytestmark = [
    pytest.mark.gpu,
]


def rand_graph(seed, n_lo=40, n_hi=220, L_hi=4):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi))
    L = int(rng.integers(1, L_hi + 1))
    p = float(rng.uniform(0.05, 0.2))
    edges = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p], np.int32).reshape(-1, 2)
    labels = rng.integers(0, L, size=n).astype(np.int32)
    return rng, n, edges, labels, L


def rand_query(rng, L, k):
    qe = set()
    for v in range(1, k):
        qe.add((int(rng.integers(0, v)), v))
    for a in range(k):
        for b in range(a + 1, k):
            if rng.random() < 0.3:
                qe.add((a, b))
    return rng.integers(0, L, size=k).astype(np.int32), np.array(sorted(qe), np.int32).reshape(-1, 2)


def check(csts, cfg):
    got, status = F.partition_many(csts, cfg)
    for c, ch, st in zip(csts, got, status):
        if c is None:
            assert st == F.FAST_ERR_INVALID and ch is None
            continue
        assert st == 0
        want = F.Chunks(c, cfg)
        assert ch.n == want.n
        assert ch.copy() == want.copy()
        assert ch.w_sum == want.w_sum
        mc = F.default_config(limit=1 << 20)
        assert F.match(c, ch, cfg=mc)["count"] == F.match(c, want, cfg=mc)["count"]
        want.close()
        ch.close()


CFGS = [dict(delta_w=1 << 20), dict(delta_w=64), dict(delta_w=8, max_chunks=64), dict(delta_w=1, max_chunks=7),
        dict(delta_w=16, sample_root=2.0, sample_deep=1.5, sample_seed=5)]


@pytest.mark.parametrize("ci", range(len(CFGS)))
@pytest.mark.parametrize("seed", range(6))
def test_random_graphs(seed, ci):
    rng, n, e, lab, L = rand_graph(8100 + seed)
    g = F.Graph(n, e, lab)
    csts = [F.Cst(g, *rand_query(rng, L, int(rng.integers(1, 7)))) for _ in range(10)]
    csts.insert(3, None)
    csts.append(F.Cst(g, np.array([L + 3, 0], np.int32), np.array([[0, 1]], np.int32)))   # W = 0
    check(csts, F.default_config(**CFGS[ci]))


def test_power_law_graph():
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    csts = []
    for k in (4, 8, 12):
        for j, kind in enumerate(("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for r in range(4):
                q = wg.query(lab, k, kind, seed=55, stream=100 * k + 10 * j + r)
                csts.append(F.Cst(g, q.labels, q.edges, F.default_config(order_rule=1)))
    for cfg in (dict(delta_w=1 << 20, max_chunks=4096), dict(delta_w=1 << 12, max_chunks=512)):
        got, status = F.partition_many(csts, F.default_config(**cfg))
        assert status.tolist() == [0] * len(csts)
        for c, ch in zip(csts, got):
            want = F.Chunks(c, F.default_config(**cfg))
            assert ch.copy() == want.copy()
            want.close()
            ch.close()


def test_batch_run_with_batched_partitions():
    """fast_batch_run with build_rule 2 (CSTs and partitions together) gives
    the counts and statuses of the per-query path."""
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = []
    for k in (4, 8, 16):
        for j, kind in enumerate(("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for r in range(6):
                q = wg.query(lab, k, kind, seed=93, stream=100 * k + 10 * j + r)
                qs.append((q.labels, q.edges))
    qs.insert(3, (np.array([0, 1, 0], np.int32), np.array([[0, 1]], np.int32)))      # disconnected
    for rule in (dict(), dict(order_rule=1, filter_rule=1)):
        base = F.default_config(limit=1 << 16, time_budget_s=60.0, max_chunks=1024, **rule)
        c0, s0 = F.Batch(g, len(qs), base).run(qs)
        both = F.Config.from_buffer_copy(base)
        both.build_rule = 2
        c2, s2 = F.Batch(g, len(qs), both).run(qs)
        assert s2.tolist() == s0.tolist() and c2.tolist() == c0.tolist(), rule
