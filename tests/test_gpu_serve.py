"""Serving with continuous batching: requests queued while a group runs are
run together as the next group (one batched build and one matcher launch);
every request's result equals the one it gets alone; admission by projected
bytes serialises requests when the budget holds only one, and rejects a
request that exceeds the whole budget."""
import time

import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    F.build()
    w = synth.er_workload()
    g = F.Graph(w.n, w.edges, w.labels)
    wg = synth.WalkGraph(w.n, w.edges)
    qs = [(q.labels, q.edges) for q in w.queries]
    for i, k in enumerate((3, 5, 6, 7, 8, 9, 10, 12)):
        q = wg.query(w.labels, k, "sparse" if i % 2 else "induced", seed=21, stream=i)
        qs.append((q.labels, q.edges))
    alone = []
    for ql, qe in qs:
        alone.append(F.match(F.Cst(g, ql, qe))["count"])
    return w, g, qs, alone


def drain(server, n, timeout_s=120.0):
    out = []
    t0 = time.time()
    while len(out) < n and time.time() - t0 < timeout_s:
        out += server.poll(256, wait_ms=50)
    return out


@pytest.mark.parametrize("seed", range(3))
def test_results_equal_alone_under_random_arrivals(env, seed):
    w, g, qs, alone = env
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(qs))
    s = F.Server(g, budget_bytes=8 << 30, cfg=F.default_config(blocks_per_sm=1), workers=4)
    ids = {}
    for i in order:
        ids[s.submit(*qs[i])] = i
        time.sleep(float(rng.uniform(0, 0.003)))
    res = drain(s, len(qs))
    s.close()
    assert len(res) == len(qs)
    for r in res:
        assert r["status"] == 0
        assert r["count"] == alone[ids[r["id"]]]
        assert r["t_arrive_ns"] <= r["t_start_ns"] <= r["t_done_ns"]


def test_requests_queued_meanwhile_run_as_one_group(env):
    w, g, qs, alone = env
    s = F.Server(g, budget_bytes=8 << 30, cfg=F.default_config(build_rule=2), workers=1)
    reps = 5
    ids = {}
    for r in range(reps):                     # all at once: the first group starts while the rest queue
        for i, q in enumerate(qs):
            ids[s.submit(*q)] = i
    res = drain(s, len(ids))
    groups, grouped = s.groups()
    s.close()
    assert len(res) == len(ids) == grouped
    assert groups < grouped / 4, (groups, grouped)
    for r in res:
        assert r["status"] == 0
        assert r["count"] == alone[ids[r["id"]]]
    # the requests of a group are admitted together and finish together
    spans = {}
    for r in res:
        spans.setdefault(r["t_start_ns"], set()).add(r["t_done_ns"])
    assert len(spans) == groups and all(len(v) == 1 for v in spans.values())


def test_budget_for_one_request_serialises(env):
    w, g, qs, alone = env
    s0 = F.Server(g, budget_bytes=1 << 40, workers=1)
    s0.close()
    # a budget that holds any single request here (16 MB of matcher scratch plus
    # well under 4 MB of CST on this 10k-vertex graph) but never two
    s = F.Server(g, budget_bytes=24 << 20, cfg=F.default_config(blocks_per_sm=1), workers=4)
    ids = {s.submit(*q): i for i, q in enumerate(qs[:8])}
    res = drain(s, 8)
    s.close()
    assert len(res) == 8 and all(r["status"] == 0 for r in res)
    for r in res:
        assert r["count"] == alone[ids[r["id"]]]
    spans = sorted((r["t_start_ns"], r["t_done_ns"]) for r in res)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1                       # never two at once


def test_request_beyond_the_budget_is_rejected(env):
    w, g, qs, alone = env
    s = F.Server(g, budget_bytes=1 << 20, workers=2)
    rid = s.submit(*qs[0])
    res = drain(s, 1)
    s.close()
    assert res[0]["id"] == rid and res[0]["status"] == F.FAST_ERR_OOM


def test_malformed_requests_come_back_invalid(env):
    import ctypes
    w, g, qs, alone = env
    bad = [
        (np.array([0, 1, 2], np.int32), np.array([[0, 1], [1, 7]], np.int32)),    # endpoint out of range
        (np.array([0, -3, 2], np.int32), np.array([[0, 1], [1, 2]], np.int32)),   # negative label
        (np.array([0, 1, 2], np.int32), np.array([[0, 1], [-1, 2]], np.int32)),   # negative endpoint
        (np.array([0, 1, 2], np.int32), np.array([[0, 1]], np.int32)),            # disconnected
        (np.array([0, 1], np.int32), np.array([[0, 0], [0, 1]], np.int32)),       # loop
    ]
    s = F.Server(g, budget_bytes=1 << 40, workers=2)
    ids = {s.submit(*q): ("bad", i) for i, q in enumerate(bad)}
    ids.update({s.submit(*q): ("good", i) for i, q in enumerate(qs[:4])})
    res = drain(s, len(ids))
    n = ctypes.c_int32(-1)
    rc = F.lib().fast_server_poll(s._h, -1, None, ctypes.byref(n), 0)
    s.close()
    assert rc == F.FAST_ERR_INVALID
    assert len(res) == len(ids)
    for r in res:
        kind, i = ids[r["id"]]
        if kind == "bad":
            assert r["status"] == F.FAST_ERR_INVALID and r["count"] == 0, (i, r)
        else:
            assert r["status"] == 0 and r["count"] == alone[i]


def test_limit_in_the_mix_matches_oracle():
    n, e, lab = synth.powerlaw_graph(seed=2000, n=200_000, m=3_200_000)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    qs = []
    L = 1 << 16
    for k in (4, 8):
        for kind in (("induced", "sparse") if k == 4 else ("dense", "sparse")):
            for q in synth.walk_queries(n, e, lab, k, 3, kind, seed=6, stream0=10 * k + (5 if kind == "sparse" else 0)):
                r = oracle.match(o, q.labels, q.edges, limit=L, budget=50_000_000)
                if r["complete"] and r["count"] == L:
                    qs.append((q.labels, q.edges))
    assert len(qs) >= 4
    s = F.Server(g, budget_bytes=16 << 30, cfg=F.default_config(limit=L, blocks_per_sm=1, max_chunks=1024,
                                                               time_budget_s=30.0), workers=4)
    ids = {s.submit(*q): i for i, q in enumerate(qs)}
    res = drain(s, len(qs))
    s.close()
    assert len(res) == len(qs)
    for r in res:
        ql, qe = qs[ids[r["id"]]]
        assert r["status"] == 0
        assert r["count"] == oracle.match(o, ql, qe, limit=L)["count"]
