"""Batched matching (one graph-replayed matcher launch for many queries)
against the oracle and against per-query launches: counts are exact and do
not depend on which other queries share the launch."""
import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def er():
    F.build()
    w = synth.er_workload()
    return w, F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)


def mixed_queries(w, seed):
    rng = np.random.default_rng(seed)
    qs = [(q.labels, q.edges) for q in w.queries]
    wg = synth.WalkGraph(w.n, w.edges)
    for i, k in enumerate((3, 5, 6, 7, 8, 9)):
        q = wg.query(w.labels, k, "sparse" if i % 2 else "induced", seed=seed, stream=i)
        qs.append((q.labels, q.edges))
    order = rng.permutation(len(qs))
    return [qs[i] for i in order]


def test_batch_counts_match_oracle(er):
    w, g, o = er
    qs = mixed_queries(w, 7)
    want = [oracle.count(o, ql, qe) for ql, qe in qs]
    b = F.Batch(g, 64)
    counts, status = b.run(qs)
    assert status.tolist() == [0] * len(qs)
    assert counts.tolist() == want
    # the same handle again (graph replay), and a different mix
    counts2, _ = b.run(qs)
    assert counts2.tolist() == want
    sub = qs[::3]
    c3, _ = b.run(sub)
    assert c3.tolist() == want[::3]


def test_batch_result_independent_of_the_mix(er):
    w, g, o = er
    qs = mixed_queries(w, 8)
    b = F.Batch(g, 64)
    alone = []
    for q in qs:
        c, s = b.run([q])
        alone.append(int(c[0]))
    together, _ = b.run(qs)
    assert together.tolist() == alone
    rev, _ = b.run(qs[::-1])
    assert rev.tolist()[::-1] == alone


def test_batch_limit_and_bad_query(er):
    w, g, o = er
    qs = mixed_queries(w, 9)
    L = 50
    b = F.Batch(g, 64, F.default_config(limit=L))
    bad = ([0, 1, 2], [[0, 1]])                       # disconnected
    counts, status = b.run(qs + [bad])
    assert status[-1] == F.FAST_ERR_INVALID and counts[-1] == 0
    want = [min(oracle.count(o, ql, qe), L) for ql, qe in qs]
    assert counts[:-1].tolist() == want and all(s == 0 for s in status[:-1])


def test_batch_autotune_keeps_results(er):
    w, g, o = er
    qs = mixed_queries(w, 10)
    want = [oracle.count(o, ql, qe) for ql, qe in qs]
    b = F.Batch(g, 64)
    best = b.autotune(qs[:8])
    assert best > 0
    counts, status = b.run(qs)
    assert counts.tolist() == want
    one, _ = F.match_batch(g, qs)
    assert one.tolist() == want


@pytest.fixture(scope="module")
def powerlaw():
    F.build()
    n, e, lab = synth.powerlaw_graph(seed=2000, n=200_000, m=3_200_000)
    return n, e, lab, F.Graph(n, e, lab), oracle.Graph(n, e, lab)


def test_batch_on_powerlaw_with_limit(powerlaw):
    n, e, lab, g, o = powerlaw
    qs = []
    L = 1 << 16
    for k in (4, 8):
        for kind in (("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for q in synth.walk_queries(n, e, lab, k, 2, kind, seed=5, stream0=10 * k + (5 if kind == "sparse" else 0)):
                r = oracle.match(o, q.labels, q.edges, limit=L, budget=50_000_000)
                if r["complete"] and r["count"] == L:
                    qs.append((q.labels, q.edges))
    assert len(qs) >= 4
    b = F.Batch(g, 16, F.default_config(limit=L, max_chunks=1024, time_budget_s=30.0))
    counts, status = b.run(qs)
    assert all(s == 0 for s in status)
    for (ql, qe), c in zip(qs, counts):
        assert c == oracle.match(o, ql, qe, limit=L)["count"]


def test_batch_limit_reached_while_items_start(powerlaw):
    """Copies of one query with a small limit: the per-query stop flag flips
    while thousands of warps are picking up items and donated runs of that
    query.  Every run must end (well inside its budget) with the exact
    limited count."""
    n, e, lab, g, o = powerlaw
    q = synth.walk_queries(n, e, lab, 4, 1, "induced", seed=5, stream0=40)[0]
    for L in (1000, 1 << 16):
        want = oracle.match(o, q.labels, q.edges, limit=L)["count"]
        b = F.Batch(g, 8, F.default_config(limit=L, max_chunks=1024, time_budget_s=20.0))
        for rep in range(6):
            nq = 1 + rep % 8 if rep < 5 else 8
            counts, status = b.run([(q.labels, q.edges)] * nq)
            assert status.tolist() == [0] * nq, (L, rep)
            assert counts.tolist() == [want] * nq, (L, rep)
            assert b.timing()["match_ms"] < 5000.0
