"""The batched CST build (fast_build_cst_batch) against the oracle and
against the per-query build.

Every CST of a batch must equal the oracle's restatement of Alg. 1 and the
workload estimate (root, t_q, order, candidate sets, tree and non-tree
lists, c_u and W), in both matching orders and under both candidate
filters, and must give the same embedding counts.  Batches mix query sizes
1 to 16, invalid queries (reported per query), labels absent from G, and
more queries than one group holds.

The file runs after the other GPU tests (its name sorts last).
"""
import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth
from helpers import compare_cst

pytestmark = pytest.mark.gpu

RULES = [dict(), dict(order_rule=1), dict(filter_rule=1), dict(order_rule=1, filter_rule=1)]


def _oracle_kw(rule):
    kw = {}
    if rule.get("order_rule") == 1:
        kw["order"] = "greedy"
    if rule.get("filter_rule") == 1:
        kw["filter"] = "nlf"
    return kw


def rand_graph(seed, n_lo=40, n_hi=220, L_hi=4):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi))
    L = int(rng.integers(1, L_hi + 1))
    p = float(rng.uniform(0.03, 0.2))
    edges = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p], np.int32).reshape(-1, 2)
    labels = rng.integers(0, L, size=n).astype(np.int32)
    return rng, n, edges, labels, L


def rand_query(rng, L, k):
    qe = set()
    for v in range(1, k):
        qe.add((int(rng.integers(0, v)), v))
    dens = float(rng.uniform(0, 0.5))
    for a in range(k):
        for b in range(a + 1, k):
            if rng.random() < dens:
                qe.add((a, b))
    ql = rng.integers(0, L, size=k).astype(np.int32)
    return ql, np.array(sorted(qe), np.int32).reshape(-1, 2)


def check_batch(g, o, qs, rule, bad=()):
    cfg = F.default_config(**rule)
    csts, status = F.build_csts(g, qs, cfg)
    assert len(csts) == len(qs)
    for i, ((ql, qe), c) in enumerate(zip(qs, csts)):
        if i in bad:
            assert status[i] == F.FAST_ERR_INVALID and c is None, i
            continue
        assert status[i] == 0 and c is not None, (i, status[i])
        compare_cst(c, oracle.Cst(o, ql, qe, **_oracle_kw(rule)), len(ql))
        lim = 1 << 20                       # min(total, limit): exact, and quick on dense one-label cases
        assert F.match(c, cfg=F.default_config(limit=lim))["count"] == oracle.match(o, ql, qe, limit=lim)["count"]
        c.close()


@pytest.mark.parametrize("rule", range(len(RULES)))
@pytest.mark.parametrize("seed", range(8))
def test_batch_random_graphs(seed, rule):
    rng, n, e, lab, L = rand_graph(7000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    qs = [rand_query(rng, L, int(rng.integers(1, 8))) for _ in range(10)]
    qs.append((np.array([L + 5, 0], np.int32), np.array([[0, 1]], np.int32)))    # a label G lacks
    qs.append((np.array([0], np.int32), np.zeros((0, 2), np.int32)))             # k = 1
    bad = {len(qs), len(qs) + 1}
    qs.append((np.array([0, 1, 0], np.int32), np.array([[0, 1]], np.int32)))     # disconnected
    qs.append((np.array([0, 1], np.int32), np.array([[0, 5]], np.int32)))        # edge out of range
    check_batch(g, o, qs, RULES[rule], bad)


@pytest.mark.parametrize("rule", range(len(RULES)))
def test_batch_er_workload(rule):
    w = synth.er_workload()
    g, o = F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)
    wg = synth.WalkGraph(w.n, w.edges)
    qs = [(q.labels, q.edges) for q in w.queries]
    for i, k in enumerate((3, 5, 6, 7, 8)):
        q = wg.query(w.labels, k, "sparse" if i % 2 else "induced", seed=31, stream=i)
        qs.append((q.labels, q.edges))
    check_batch(g, o, qs, RULES[rule])


@pytest.mark.parametrize("rule", range(len(RULES)))
@pytest.mark.parametrize("seed", range(4))
def test_small_batches_build_without_round_trips(seed, rule):
    """Batches of up to 8 queries build their top-down pass with no host
    round trip (arrays sized by host-known bounds, real sizes read on the
    device): the CSTs equal the oracle's, and the build waits on the host at
    most six times whatever the query size; a batch of nine fetches every
    level's sizes and gives the same CSTs."""
    rng, n, e, lab, L = rand_graph(7100 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    qs = [rand_query(rng, L, int(rng.integers(2, 8))) for _ in range(9)]
    for size in (1, 3, 8):
        check_batch(g, o, qs[:size], RULES[rule])
        csts, status = F.build_csts(g, qs[:size], F.default_config(**RULES[rule]))
        assert F.last_build_round_trips() <= 6, size
        for c in csts:
            c.close()
    cfg = F.default_config(**RULES[rule])
    csts, status = F.build_csts(g, qs, cfg)
    kmax = max(len(ql) for ql, _ in qs)
    assert F.last_build_round_trips() >= 2 * (kmax - 1)
    small, _ = F.build_csts(g, qs[:8], cfg)
    for a, b in zip(small, csts[:8]):
        _same_cst(a, b)
        a.close()
    for c in csts:
        c.close()


def _same_cst(a, b):
    """Two CSTs of the same query from the library: equal arrays (W's
    float64 twin within rounding, its sums being atomics)."""
    assert a.root == b.root and a.order.tolist() == b.order.tolist() and a.parent.tolist() == b.parent.tolist()
    assert a.ncand.tolist() == b.ncand.tolist() and a.W == b.W
    assert abs(a.Wf - b.Wf) <= 1e-9 * max(1.0, abs(b.Wf))
    for u in range(a.k):
        assert np.array_equal(a.candidates(u), b.candidates(u))
        assert np.array_equal(a.workload(u), b.workload(u))
        if a.parent[u] >= 0:
            for x, y in zip(a.tree_lists(u), b.tree_lists(u)):
                assert np.array_equal(x, y)
    na, nb = a.nontree(), b.nontree()
    assert len(na) == len(nb)
    for x, y in zip(na, nb):
        assert x[:2] == y[:2] and np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])


def test_batch_powerlaw_equals_per_query():
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = []
    for k in (4, 8, 12, 16):
        for j, kind in enumerate(("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for r in range(5):
                q = wg.query(lab, k, kind, seed=77, stream=100 * k + 10 * j + r)
                qs.append((q.labels, q.edges))
    for rule in RULES:
        cfg = F.default_config(**rule)
        csts, status = F.build_csts(g, qs, cfg)
        assert status.tolist() == [0] * len(qs)
        for (ql, qe), c in zip(qs, csts):
            one = F.Cst(g, ql, qe, cfg)
            _same_cst(c, one)
            lim = F.default_config(limit=1 << 16, **rule)
            assert F.match(c, cfg=lim)["count"] == F.match(one, cfg=lim)["count"]
            one.close()
            c.close()


def test_small_batches_powerlaw_equal_per_query():
    """The bounded top-down pass on a power-law graph with hubs, batches of
    one to eight queries of up to 16 vertices: every CST equals the one the
    per-query build gives."""
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = []
    for k in (4, 8, 12, 16):
        for r in range(3):
            kind = ("induced", "sparse", "induced" if k == 4 else "dense")[r]
            q = wg.query(lab, k, kind, seed=78, stream=10 * k + r)
            qs.append((q.labels, q.edges))
    wg.close()
    cfg = F.default_config(filter_rule=1, order_rule=1)
    for lo, hi in ((0, 1), (1, 4), (4, 12)):
        csts, status = F.build_csts(g, qs[lo:hi], cfg)
        assert status.tolist() == [0] * (hi - lo)
        assert F.last_build_round_trips() <= 6
        for (ql, qe), c in zip(qs[lo:hi], csts):
            one = F.Cst(g, ql, qe, cfg)
            _same_cst(c, one)
            one.close()
            c.close()


def test_batch_more_than_one_group():
    w = synth.er_workload()
    g, o = F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)
    wg = synth.WalkGraph(w.n, w.edges)
    qs = []
    for i in range(1100):
        q = wg.query(w.labels, 2 + i % 5, "sparse" if i % 2 else "induced", seed=41, stream=i)
        qs.append((q.labels, q.edges))
    csts, status = F.build_csts(g, qs)
    assert status.tolist() == [0] * len(qs)
    for i in list(range(0, 1100, 97)) + [1023, 1024, 1099]:
        ql, qe = qs[i]
        compare_cst(csts[i], oracle.Cst(o, ql, qe), len(ql))
    for i, c in enumerate(csts):
        ql, qe = qs[i]
        assert c.W == oracle.Cst(o, ql, qe).workload()[1]
        c.close()


def test_batch_empty_and_all_invalid():
    w = synth.er_workload()
    g = F.Graph(w.n, w.edges, w.labels)
    csts, status = F.build_csts(g, [])
    assert csts == [] and status.size == 0
    csts, status = F.build_csts(g, [(np.array([0, 1, 2], np.int32), np.array([[0, 1]], np.int32))])
    assert csts == [None] and status.tolist() == [F.FAST_ERR_INVALID]


def test_batch_run_with_the_batched_build():
    """fast_batch_run with build_rule 1 gives the counts and statuses of the
    per-query build, invalid queries included."""
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = []
    for k in (4, 8, 16):
        for j, kind in enumerate(("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for r in range(8):
                q = wg.query(lab, k, kind, seed=91, stream=100 * k + 10 * j + r)
                qs.append((q.labels, q.edges))
    qs.insert(5, (np.array([0, 1, 0], np.int32), np.array([[0, 1]], np.int32)))      # disconnected
    for rule in RULES:
        base = F.default_config(limit=1 << 16, time_budget_s=60.0, **rule)
        c0, s0 = F.Batch(g, len(qs), base).run(qs)
        one = F.Config.from_buffer_copy(base)
        one.build_rule = 1
        c1, s1 = F.Batch(g, len(qs), one).run(qs)
        assert s1.tolist() == s0.tolist() and c1.tolist() == c0.tolist(), rule
        assert s0[5] == F.FAST_ERR_INVALID


def test_batch_create_rejects_unknown_build_rule():
    w = synth.er_workload()
    g = F.Graph(w.n, w.edges, w.labels)
    with pytest.raises(F.FastError):
        F.Batch(g, 4, F.default_config(build_rule=3))


def test_refine_rule_needs_the_batched_build():
    """The per-query build and the threaded batch reject refine rule 2 before
    any device work; rule 1 (the fixpoint) is the oracle's only."""
    w = synth.er_workload()
    g = F.Graph(w.n, w.edges, w.labels)
    q = w.queries[0]
    with pytest.raises(F.FastError):
        F.Cst(g, q.labels, q.edges, F.default_config(refine_rule=2))
    with pytest.raises(F.FastError):
        F.Batch(g, 4, F.default_config(refine_rule=2))
    with pytest.raises(F.FastError):
        F.Batch(g, 4, F.default_config(refine_rule=1, build_rule=1))
