"""The warp-specialised matcher (fast_config.matcher_rule 1: expander warps
hand last-position extensions to validator warps through a ring in shared
memory, the task-generator separation of Sec. V-D) against the oracle and
against the fused kernel.

Counts equal the oracle on random graphs in both matching orders, with one
to seven validator warps per CTA, with and without a partition; the floor
of the bytes read equals the oracle's (the split between expanders and
validators reads exactly what the fused search reads); a hub that makes
idle warps steal work all the time, a tiny ring of donated runs, the
enumeration limit, the time budget, and the batched launch (many queries,
one graph-replayed launch) give the fused kernel's results.
"""
import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth
from test_gpu_parity import rand_case

pytestmark = pytest.mark.gpu


def ws(**kw):
    return F.default_config(matcher_rule=1, **kw)


def _oracle_balg(o, oc, ql, qe):
    k = len(ql)
    allow = {u: oc.cand(u).tolist() for u in range(k)}
    pos = {int(u): i for i, u in enumerate(oc.order)}
    par = [0] + [pos[int(oc.parent[int(oc.order[i])])] for i in range(1, k)]
    return oracle.match(o, ql, qe, order=oc.order, par=par, allow=allow, want_balg=True)


@pytest.mark.parametrize("seed", range(16))
def test_counts_and_floor_match_oracle(seed):
    n, e, lab, ql, qe = rand_case(6100 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    order = ("path", "greedy")[seed % 2]
    cfg = F.default_config(order_rule=seed % 2)
    gc, oc = F.Cst(g, ql, qe, cfg), oracle.Cst(o, ql, qe, order=order)
    want = _oracle_balg(o, oc, ql, qe)
    for v in (1, 4, 7):
        r = F.match(gc, cfg=ws(validators=v, order_rule=seed % 2))
        assert r["count"] == want["count"], v
        assert F.last_match_floor_bytes() == want["balg"], v
    ch = F.Chunks(gc, F.default_config(delta_w=max(1, gc.W // 32)))
    assert F.match(gc, ch, cfg=ws())["count"] == want["count"]


def test_skewed_tree_and_tiny_rings():
    rng = np.random.default_rng(21)
    n = 3000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(6000, 2)) if x[0] != x[1]]
    e = np.array(e, np.int32)
    lab = np.zeros(n, np.int32)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    for qe in ([[0, 1], [1, 2], [2, 3]], [[0, 1], [1, 2], [0, 2], [2, 3]], [[0, 1], [1, 2], [2, 3], [3, 4]]):
        ql = np.zeros(int(np.max(qe)) + 1, np.int32)
        want = oracle.count(o, ql, qe)
        cst = F.Cst(g, ql, qe)
        for cells in (0, 1, 7):
            assert F.match(cst, cfg=ws(queue_cells=cells))["count"] == want
        lim = max(1, want // 3)
        assert F.match(cst, cfg=ws(limit=lim))["count"] == min(want, lim)
        assert F.match(cst, F.Chunks(cst, F.default_config(delta_w=max(1, cst.W // 64))), cfg=ws())["count"] == want


def test_time_budget_reports_timeout():
    n = 20_000
    e = synth.chung_lu_edges(n, 200_000, 2.1, 5)
    g = F.Graph(n, e, np.zeros(n, np.int32))
    cst = F.Cst(g, np.zeros(6, np.int32), [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]])
    r = F.match(cst, cfg=ws(time_budget_s=0.05), check=False)
    assert r["status"] == F.FAST_ERR_TIMEOUT


def test_batched_launch_equals_fused_and_oracle():
    w = synth.er_workload()
    g, o = F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)
    wg = synth.WalkGraph(w.n, w.edges)
    qs = [(q.labels, q.edges) for q in w.queries]
    for k in (3, 5, 6, 7):
        for j, kind in enumerate(("induced", "sparse")):
            q = wg.query(w.labels, k, kind, 91, 10 * k + j)
            qs.append((q.labels, q.edges))
    wg.close()
    want = [oracle.count(o, ql, qe) for ql, qe in qs]
    fused, _ = F.Batch(g, len(qs), F.default_config()).run(qs)
    for v in (0, 2, 6):
        b = F.Batch(g, len(qs), ws(validators=v))
        counts, status = b.run(qs)
        assert status.tolist() == [0] * len(qs)
        assert counts.tolist() == want == fused.tolist(), v
        counts2, _ = b.run(qs[::2])                       # graph replay, another mix
        assert counts2.tolist() == want[::2]


def test_powerlaw_limit_counts_equal_fused():
    n, e, lab = synth.powerlaw_graph(seed=2000, n=200_000, m=3_200_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = synth.mixed_queries(wg, lab, (4, 8, 16), 6, 3000)
    wg.close()
    base = dict(limit=1 << 18, order_rule=1, filter_rule=1, time_budget_s=60.0, build_rule=2)
    fused, s0 = F.Batch(g, len(qs), F.default_config(**base)).run(qs)
    spec, s1 = F.Batch(g, len(qs), ws(**base)).run(qs)
    assert s0.tolist() == s1.tolist() == [0] * len(qs)
    assert spec.tolist() == fused.tolist()
    for ql, qe in qs[:6]:
        cst = F.Cst(g, ql, qe, F.default_config(order_rule=1, filter_rule=1))
        ch = F.Chunks(cst, F.default_config(max_chunks=1024))
        assert F.match(cst, ch, cfg=ws(limit=1 << 18))["count"] == F.match(cst, ch, cfg=F.default_config(limit=1 << 18))["count"]
