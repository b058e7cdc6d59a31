"""Failure injection on the host: every device allocation of the library can
be made to fail (fast_inject_alloc_failure), and each failure must come back
as FAST_ERR_OOM from the call that made it -- as an exception, or as a
query's status in a batch -- with nothing left half done: the calls right
after it work and give the oracle's results.  The failure is an error code
from the allocation call; no test faults, traps or hangs the GPU.

Each sweep fails allocation n of one pipeline for n = 0, 1, 2, ... until the
pipeline gets through without reaching the injected failure.
"""

import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth

pytestmark = [
    pytest.mark.gpu,
]

LIMIT = 5000


@pytest.fixture(scope="module")
def er():
    F.build()
    w = synth.er_workload()
    return w, F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)


def sweep(run, check):
    """Fails allocation n of run() for n = 0, 1, ... until run() makes fewer
    than n + 1 allocations; returns that n (the pipeline's allocation count).
    A failed run raises FAST_ERR_OOM or reports it in its result (check
    accepts that); the run right after it works."""
    for n in range(LIMIT):
        F.inject_alloc_failure(n)
        try:
            out = run()
        except F.FastError as e:
            assert F.inject_alloc_failure(-1) == -1, n           # the injected failure, not another
            assert e.code == F.FAST_ERR_OOM, (n, str(e))
            check(run())
            continue
        left = F.inject_alloc_failure(-1)
        check(out)
        if left >= 0:
            return n                                             # never reached: done
        check(run())
    raise AssertionError("the pipeline kept failing")


def test_per_query_pipeline(er):
    w, g, o = er
    q = w.queries[0]
    want = oracle.count(o, q.labels, q.edges)

    def run():
        cst = F.Cst(g, q.labels, q.edges, F.default_config(filter_rule=1))
        ch = F.Chunks(cst, F.default_config(delta_w=64))
        r = F.match(cst, ch, k=8)
        ch.close()
        cst.close()
        return r["count"]

    def check(c):
        assert c == want

    assert sweep(run, check) > 5


def test_graph_loader():
    F.build()
    n, e, lab = synth.powerlaw_graph(seed=2000, n=20_000, m=200_000)

    def run():
        g = F.Graph(n, e, lab)
        inf = g.info()
        g.close()
        return inf["nadj"]

    def check(nadj):
        assert nadj == 2 * e.shape[0]

    assert sweep(run, check) > 3


def test_batched_paths(er):
    w, g, o = er
    qs = [(q.labels, q.edges) for q in w.queries]
    want = [oracle.count(o, ql, qe) for ql, qe in qs]

    for rule in (0, 1, 2):
        cfg = F.default_config(build_rule=rule)

        def run():
            b = F.Batch(g, len(qs), cfg)
            try:
                return b.run(qs)
            finally:
                b.close()

        def check(out):
            counts, status = out
            for i, (c, s) in enumerate(zip(counts.tolist(), status.tolist())):
                # a query whose own build met the injected failure reports it
                assert s in (0, F.FAST_ERR_OOM), (i, s)
                if s == 0:
                    assert c == want[i], (i, c, want[i])

        sweep(run, check)
        counts, status = F.Batch(g, len(qs), cfg).run(qs)
        assert status.tolist() == [0] * len(qs) and counts.tolist() == want


def test_server(er):
    w, g, o = er
    qs = [(q.labels, q.edges) for q in w.queries[:4]]
    want = [oracle.count(o, ql, qe) for ql, qe in qs]
    for n in range(0, 400, 7):
        s = F.Server(g, budget_bytes=1 << 40, workers=2)
        F.inject_alloc_failure(n)
        try:
            ids = {s.submit(*q): i for i, q in enumerate(qs)}
            res = []
            while len(res) < len(qs):
                res += s.poll(16, wait_ms=100)
        finally:
            F.inject_alloc_failure(-1)
            s.close()
        for r in res:
            assert r["status"] in (0, F.FAST_ERR_OOM)
            if r["status"] == 0:
                assert r["count"] == want[ids[r["id"]]]
