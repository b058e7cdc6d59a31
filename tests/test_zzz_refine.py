"""Refine rule 2 (the bottom-up pass with the non-tree neighbour test) in
the batched CST build, against the oracle's restatement of the same rule:
every CST array, in both orders and under both filters, and the same
embedding counts as the paper's single pass.
"""

import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth
from helpers import compare_cst

pytestmark = [
    pytest.mark.gpu,
]

RULES = [dict(), dict(order_rule=1), dict(filter_rule=1), dict(order_rule=1, filter_rule=1)]


def _kw(rule):
    kw = {"refine": "once_nt"}
    if rule.get("order_rule") == 1:
        kw["order"] = "greedy"
    if rule.get("filter_rule") == 1:
        kw["filter"] = "nlf"
    return kw


def rand_case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 200))
    L = int(rng.integers(1, 4))
    p = float(rng.uniform(0.05, 0.2))
    edges = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p], np.int32).reshape(-1, 2)
    labels = rng.integers(0, L, size=n).astype(np.int32)
    qs = []
    for _ in range(8):
        k = int(rng.integers(2, 7))
        qe = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        for a in range(k):
            for b in range(a + 1, k):
                if rng.random() < 0.4:
                    qe.add((a, b))
        qs.append((rng.integers(0, L, size=k).astype(np.int32), np.array(sorted(qe), np.int32).reshape(-1, 2)))
    return n, edges, labels, qs


@pytest.mark.parametrize("rule", range(len(RULES)))
@pytest.mark.parametrize("seed", range(8))
def test_random_graphs(seed, rule):
    n, e, lab, qs = rand_case(9100 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    cfg = F.default_config(refine_rule=2, **RULES[rule])
    csts, status = F.build_csts(g, qs, cfg)
    for (ql, qe), c, st in zip(qs, csts, status):
        assert st == 0
        compare_cst(c, oracle.Cst(o, ql, qe, **_kw(RULES[rule])), len(ql))
        assert F.match(c)["count"] == oracle.count(o, ql, qe)
        c.close()


def test_batch_counts_equal_the_single_pass():
    n, e, lab = synth.powerlaw_graph(seed=2000, n=50_000, m=600_000)
    g = F.Graph(n, e, lab)
    wg = synth.WalkGraph(n, e)
    qs = []
    for k in (4, 8, 16):
        for j, kind in enumerate(("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for r in range(6):
                q = wg.query(lab, k, kind, seed=97, stream=100 * k + 10 * j + r)
                qs.append((q.labels, q.edges))
    base = F.default_config(limit=1 << 16, time_budget_s=60.0, order_rule=1, filter_rule=1)
    c0, s0 = F.Batch(g, len(qs), base).run(qs)
    ref = F.Config.from_buffer_copy(base)
    ref.build_rule = 1
    ref.refine_rule = 2
    c2, s2 = F.Batch(g, len(qs), ref).run(qs)
    assert s2.tolist() == s0.tolist() and c2.tolist() == c0.tolist()
