"""Parity of the CUDA path (through the C ABI) with the oracle, element by
element on seeded inputs.  Integer work: bit-exact.  The float64 workload
estimate: relative 1e-9 (its uint64 twin is exact)."""
import itertools
import math

import numpy as np
import pytest

import oracle
import paper_2102_10768_gb300 as F
import synth
from helpers import compare_cst, csr_by_label, gpu_chunks_global, sorted_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    F.build()
    F.lib()


@pytest.fixture(scope="module")
def er():
    w = synth.er_workload()
    return w, F.Graph(w.n, w.edges, w.labels), oracle.Graph(w.n, w.edges, w.labels)


def rand_case(seed, n_lo=30, n_hi=200, k_hi=7, L_hi=4):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi))
    L = int(rng.integers(1, L_hi + 1))
    p = float(rng.uniform(0.03, 0.2))
    edges = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p], np.int32).reshape(-1, 2)
    labels = rng.integers(0, L, size=n).astype(np.int32)
    k = int(rng.integers(1, k_hi + 1))
    qe = set()
    for v in range(1, k):
        qe.add((int(rng.integers(0, v)), v))
    for a in range(k):
        for b in range(a + 1, k):
            if rng.random() < float(rng.uniform(0, 0.5)):
                qe.add((a, b))
    ql = rng.integers(0, L, size=k).astype(np.int32)
    return n, edges, labels, ql, np.array(sorted(qe), np.int32).reshape(-1, 2)


# ------------------------------------------------------------------ loader

def _csr_equal(n, edges, labels):
    g = F.Graph(n, edges, labels)
    o = oracle.Graph(n, edges, labels)
    goff, gcol = g.csr()
    ooff, ocol = csr_by_label(*o.csr(), labels)
    assert np.array_equal(goff, ooff)
    assert np.array_equal(gcol, ocol)
    inf = g.info()
    assert inf["nadj"] == ocol.shape[0]
    deg = np.diff(ooff)
    assert inf["max_degree"] == (int(deg.max()) if n else 0)
    assert inf["num_labels"] == int(np.max(labels)) + 1


def test_loader_er(er):
    w, g, o = er
    goff, gcol = g.csr()
    ooff, ocol = csr_by_label(*o.csr(), w.labels)
    assert np.array_equal(goff, ooff) and np.array_equal(gcol, ocol)


def test_loader_powerlaw_small():
    e = synth.chung_lu_edges(50_000, 400_000, 2.1, 77)
    lab = synth.labels_zipf(50_000, 16, 77)
    _csr_equal(50_000, e, lab)


def test_loader_duplicates_loops_isolated():
    rng = np.random.default_rng(3)
    n = 3000
    e = rng.integers(0, n // 2, size=(20000, 2)).astype(np.int32)    # upper half isolated
    e[::7, 1] = e[::7, 0]                                             # self loops
    e = np.concatenate([e, e[:5000, ::-1]])                           # reversed repeats
    _csr_equal(n, e, rng.integers(0, 5, size=n).astype(np.int32))


def test_loader_tiny():
    _csr_equal(1, np.zeros((0, 2), np.int32), np.zeros(1, np.int32))
    _csr_equal(2, np.array([[0, 1]], np.int32), np.array([3, 0], np.int32))


def test_loader_rejects_bad_input():
    with pytest.raises(F.FastError) as ei:
        F.Graph(4, np.array([[0, 4]], np.int32), np.zeros(4, np.int32))
    assert ei.value.code == F.FAST_ERR_INVALID
    with pytest.raises(F.FastError) as ei:
        F.Graph(4, np.array([[0, 1]], np.int32), np.array([0, -1, 0, 0], np.int32))
    assert ei.value.code == F.FAST_ERR_INVALID


# --------------------------------------------------------------------- CST

def test_cst_er_queries(er):
    w, g, o = er
    for q in w.queries:
        compare_cst(F.Cst(g, q.labels, q.edges), oracle.Cst(o, q.labels, q.edges), q.k)


@pytest.mark.parametrize("seed", range(40))
def test_cst_random(seed):
    n, e, lab, ql, qe = rand_case(1000 + seed)
    g = F.Graph(n, e, lab)
    o = oracle.Graph(n, e, lab)
    compare_cst(F.Cst(g, ql, qe), oracle.Cst(o, ql, qe), len(ql))


def test_cst_rejects_bad_query(er):
    w, g, o = er
    with pytest.raises(F.FastError):
        F.Cst(g, [0, 1, 2], [[0, 1]])                      # disconnected
    with pytest.raises(F.FastError):
        F.Cst(g, [0, 1], [[0, 0]])                         # loop
    with pytest.raises(F.FastError):
        F.Cst(g, list(range(33)), [[i, i + 1] for i in range(32)])   # too large


# ------------------------------------------------------------------- match

def _check_match(g, o, ql, qe, kemb_extra=3):
    cst = F.Cst(g, ql, qe)
    want = oracle.match(o, ql, qe, max_emb=1 << 20)
    assert want["complete"]
    r = F.match(cst)
    assert r["count"] == want["count"]
    if want["count"] <= 200_000:
        kk = want["count"] + kemb_extra
        r2 = F.match(cst, k=kk)
        assert r2["count"] == want["count"] and r2["written"] == want["count"]
        rows = sorted_rows(r2["emb"][:r2["written"]].astype(np.int32))
        assert np.array_equal(rows, want["emb"])
    return want["count"]


def test_match_er_queries(er):
    w, g, o = er
    total = 0
    for q in w.queries:
        total += _check_match(g, o, q.labels, q.edges)
        # the walk's own vertices always form an embedding
    assert total > 0


@pytest.mark.parametrize("seed", range(60))
def test_match_random(seed):
    n, e, lab, ql, qe = rand_case(2000 + seed)
    _check_match(F.Graph(n, e, lab), oracle.Graph(n, e, lab), ql, qe)


@pytest.mark.parametrize("seed", range(20))
def test_match_brute_force_tiny(seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(3, 8))
    e = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.6], np.int32).reshape(-1, 2)
    lab = rng.integers(0, 2, size=n).astype(np.int32)
    k = int(rng.integers(1, min(n, 5) + 1))
    qe = np.array([(int(rng.integers(0, v)), v) for v in range(1, k)] +
                  [(a, b) for a in range(k) for b in range(a + 2, k) if rng.random() < 0.4], np.int32).reshape(-1, 2)
    ql = rng.integers(0, 2, size=k).astype(np.int32)
    want = oracle.brute_force(n, e, lab, ql, qe)
    cst = F.Cst(F.Graph(n, e, lab), ql, qe)
    r = F.match(cst, k=len(want) + 2)
    assert r["count"] == len(want)
    got = [tuple(int(x) for x in row) for row in sorted_rows(r["emb"][:r["written"]].astype(np.int64))]
    assert got == want


@pytest.mark.parametrize("n,k", [(6, 1), (6, 3), (8, 5), (9, 6), (12, 4)])
def test_clique_in_complete_graph_gpu(n, k):
    e = np.array(list(itertools.combinations(range(n), 2)), np.int32)
    g = F.Graph(n, e, np.zeros(n, np.int32))
    qe = np.array(list(itertools.combinations(range(k), 2)), np.int32).reshape(-1, 2)
    assert F.match(F.Cst(g, np.zeros(k, np.int32), qe))["count"] == math.perm(n, k)


@pytest.mark.parametrize("n,L", [(3, 2), (10, 4), (50, 9), (500, 30)])
def test_path_in_cycle_gpu(n, L):
    e = np.array([[i, (i + 1) % n] for i in range(n)], np.int32)
    g = F.Graph(n, e, np.zeros(n, np.int32))
    qe = np.array([[i, i + 1] for i in range(L)], np.int32)
    assert F.match(F.Cst(g, np.zeros(L + 1, np.int32), qe))["count"] == 2 * n


def test_degenerate_queries(er):
    w, g, o = er
    # a label G does not carry: empty candidate set, count 0
    cst = F.Cst(g, [99, 0], [[0, 1]])
    assert cst.W == 0 and F.match(cst)["count"] == 0
    # one vertex: every vertex with the label
    cst = F.Cst(g, [3], np.zeros((0, 2), np.int32))
    assert F.match(cst)["count"] == int((w.labels == 3).sum())
    # all labels equal: injectivity carries the whole check
    _check_match(g, o, [1, 1, 1], [[0, 1], [1, 2]])
    _check_match(g, o, [2, 2, 2], [[0, 1], [1, 2], [0, 2]])


# ------------------------------------------- matching order: greedy rule

GREEDY = dict(order_rule=1)


@pytest.mark.parametrize("seed", range(20))
def test_cst_random_greedy_order(seed):
    """The greedy order (fast_config.order_rule = 1) against the oracle's
    restatement of the same rule: root, t_q, order, candidate sets, tree and
    non-tree lists (their direction follows the order), workload."""
    n, e, lab, ql, qe = rand_case(1000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    compare_cst(F.Cst(g, ql, qe, F.default_config(**GREEDY)), oracle.Cst(o, ql, qe, order="greedy"), len(ql))


@pytest.mark.parametrize("seed", range(20))
def test_match_random_greedy_order(seed):
    """Counts and embedding sets do not depend on the order."""
    n, e, lab, ql, qe = rand_case(2000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    cst = F.Cst(g, ql, qe, F.default_config(**GREEDY))
    want = oracle.match(o, ql, qe, max_emb=1 << 20)
    r = F.match(cst)
    assert r["count"] == want["count"]
    if want["count"] <= 200_000:
        r2 = F.match(cst, k=want["count"] + 3)
        assert np.array_equal(sorted_rows(r2["emb"][:r2["written"]].astype(np.int32)), want["emb"])


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("rule,name", [(2, "bfs"), (3, "mincand")])
def test_cst_and_counts_bfs_and_fewest_candidate_orders(seed, rule, name):
    """Order rules 2 (BFS order of t_q) and 3 (fewest candidates first):
    every CST array equals the oracle's restatement, and the counts the
    oracle's."""
    n, e, lab, ql, qe = rand_case(2400 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    cfg = F.default_config(order_rule=rule)
    gc = F.Cst(g, ql, qe, cfg)
    compare_cst(gc, oracle.Cst(o, ql, qe, order=name), len(ql))
    assert F.match(gc, F.Chunks(gc, F.default_config(delta_w=max(1, gc.W // 16))))["count"] == oracle.count(o, ql, qe)
    csts, st = F.build_csts(g, [(ql, qe)], cfg)                  # the batched build, same rules
    compare_cst(csts[0], oracle.Cst(o, ql, qe, order=name), len(ql))


def test_er_queries_greedy_order(er):
    w, g, o = er
    for q in w.queries:
        gc = F.Cst(g, q.labels, q.edges, F.default_config(**GREEDY))
        compare_cst(gc, oracle.Cst(o, q.labels, q.edges, order="greedy"), q.k)
        assert F.match(gc)["count"] == oracle.count(o, q.labels, q.edges)


@pytest.mark.parametrize("seed", range(8))
def test_partition_matches_oracle_greedy_order(seed):
    n, e, lab, ql, qe = rand_case(4000 + seed, n_lo=60, n_hi=250, k_hi=6, L_hi=3)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc, oc = F.Cst(g, ql, qe, F.default_config(**GREEDY)), oracle.Cst(o, ql, qe, order="greedy")
    if gc.W == 0:
        return
    total = oracle.count(o, ql, qe)
    for div in (7, 50):
        delta = max(1, gc.W // div)
        ch = F.Chunks(gc, F.default_config(delta_w=delta, sample_seed=seed, **GREEDY))
        assert gpu_chunks_global(gc, ch) == oc.partition(delta, 0.0, 0.0, seed)
        assert F.match(gc, ch)["count"] == total


def test_order_rule_rejected_when_unknown(er):
    w, g, o = er
    q = w.queries[0]
    with pytest.raises(F.FastError) as ei:
        F.Cst(g, q.labels, q.edges, F.default_config(order_rule=4))
    assert ei.value.code == F.FAST_ERR_INVALID
    for bad in (-1, 4):
        csts, status = F.build_csts(g, [(q.labels, q.edges)], F.default_config(order_rule=bad))
        assert status.tolist() == [F.FAST_ERR_INVALID] and csts == [None]


# ------------------------------------ candidate filter: label frequencies

NLF = dict(filter_rule=1)


@pytest.mark.parametrize("seed", range(20))
def test_cst_random_label_frequency_filter(seed):
    """filter_rule 1 against the oracle's restatement: every CST array (the
    root may change, since it follows the filtered counts), in both orders."""
    n, e, lab, ql, qe = rand_case(1000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    compare_cst(F.Cst(g, ql, qe, F.default_config(**NLF)), oracle.Cst(o, ql, qe, filter="nlf"), len(ql))
    compare_cst(F.Cst(g, ql, qe, F.default_config(order_rule=1, **NLF)),
                oracle.Cst(o, ql, qe, order="greedy", filter="nlf"), len(ql))


@pytest.mark.parametrize("seed", range(20))
def test_match_random_label_frequency_filter(seed):
    n, e, lab, ql, qe = rand_case(2000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    cst = F.Cst(g, ql, qe, F.default_config(order_rule=1, **NLF))
    want = oracle.match(o, ql, qe, max_emb=1 << 20)
    assert F.match(cst)["count"] == want["count"]
    if want["count"] <= 200_000:
        r2 = F.match(cst, k=want["count"] + 3)
        assert np.array_equal(sorted_rows(r2["emb"][:r2["written"]].astype(np.int32)), want["emb"])


def test_er_queries_label_frequency_filter(er):
    w, g, o = er
    for q in w.queries:
        gc = F.Cst(g, q.labels, q.edges, F.default_config(**NLF))
        compare_cst(gc, oracle.Cst(o, q.labels, q.edges, filter="nlf"), q.k)
        assert F.match(gc)["count"] == oracle.count(o, q.labels, q.edges)


@pytest.mark.parametrize("seed", range(6))
def test_partition_matches_oracle_label_frequency_filter(seed):
    n, e, lab, ql, qe = rand_case(4000 + seed, n_lo=60, n_hi=250, k_hi=6, L_hi=3)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc, oc = F.Cst(g, ql, qe, F.default_config(**NLF)), oracle.Cst(o, ql, qe, filter="nlf")
    if gc.W == 0:
        return
    total = oracle.count(o, ql, qe)
    delta = max(1, gc.W // 20)
    ch = F.Chunks(gc, F.default_config(delta_w=delta, sample_seed=seed, **NLF))
    assert gpu_chunks_global(gc, ch) == oc.partition(delta, 0.0, 0.0, seed)
    assert F.match(gc, ch)["count"] == total


def test_filter_rule_rejected_when_unknown(er):
    w, g, o = er
    q = w.queries[0]
    with pytest.raises(F.FastError) as ei:
        F.Cst(g, q.labels, q.edges, F.default_config(filter_rule=2))
    assert ei.value.code == F.FAST_ERR_INVALID


# --------------------------------------------------------------- partition

@pytest.mark.parametrize("seed", range(15))
def test_partition_matches_oracle(seed):
    n, e, lab, ql, qe = rand_case(4000 + seed, n_lo=60, n_hi=250, k_hi=6, L_hi=3)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc, oc = F.Cst(g, ql, qe), oracle.Cst(o, ql, qe)
    if gc.W == 0:
        return
    for div, cr, cd in ((7, 0.0, 0.0), (50, 0.0, 0.0), (40, 3.0, 1.5)):
        delta = max(1, gc.W // div)
        cfg = F.default_config(delta_w=delta, sample_root=cr, sample_deep=cd, sample_seed=seed)
        ch = F.Chunks(gc, cfg)
        want = oc.partition(delta, cr, cd, seed)
        got = gpu_chunks_global(gc, ch)
        assert got == want                       # same chunks, same level order
        # per-chunk counts against the enumerator restricted to each chunk
        import torch
        cc = torch.zeros(max(ch.n, 1), dtype=torch.int64, device="cuda")
        r = F.match(gc, ch, chunk_counts=cc)
        counts = cc.cpu().numpy()[:ch.n].astype(np.uint64)
        by_id = {c[-1]: int(counts[i]) for i, c in enumerate(ch.copy())}
        tot = 0
        for (j, pre, a, b, w, i) in want:
            c = oracle.count(o, ql, qe, allow=oc.chunk_allow(j, pre, a, b))
            assert by_id[i] == c
            assert c <= w
            tot += c
        assert r["count"] == tot
        if cr <= 0:
            assert tot == oracle.count(o, ql, qe)


# ----------------------------------------------------------------- counters

@pytest.mark.parametrize("seed", range(12))
def test_stats_match_oracle(seed):
    n, e, lab, ql, qe = rand_case(5000 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc, oc = F.Cst(g, ql, qe), oracle.Cst(o, ql, qe)
    k = len(ql)
    allow = {u: oc.cand(u).tolist() for u in range(k)}
    pos = {int(u): i for i, u in enumerate(oc.order)}
    par = [0] + [pos[int(oc.parent[int(oc.order[i])])] for i in range(1, k)]
    want = oracle.match(o, ql, qe, order=oc.order, par=par, allow=allow, want_depth=True, want_balg=True)
    b, depth = F.match_stats(gc)
    assert depth.tolist() == want["depth"].tolist()
    # the floor is exact; the bytes requested lie between floor and ceiling
    assert F.last_match_floor_bytes() == want["balg"]
    assert want["balg"] <= b <= want["balg_max"]


def _oracle_bytes(o, oc, ql, qe):
    k = len(ql)
    allow = {u: oc.cand(u).tolist() for u in range(k)}
    pos = {int(u): i for i, u in enumerate(oc.order)}
    par = [0] + [pos[int(oc.parent[int(oc.order[i])])] for i in range(1, k)]
    return oracle.match(o, ql, qe, order=oc.order, par=par, allow=allow, want_balg=True)


@pytest.mark.parametrize("seed", range(12))
def test_timed_matcher_bytes_match_oracle(seed):
    """The bytes of the timed matcher variant (no counting pass, the one the
    bench times), in both matching orders and both filters: its floor equals
    the oracle's exactly, with work donated between warps or not, and its
    requested bytes lie between the oracle's floor and ceiling."""
    import torch
    n, e, lab, ql, qe = rand_case(5200 + seed)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    for order, filt in (("path", "ldf"), ("greedy", "nlf")):
        cfg = F.default_config(order_rule=1 if order == "greedy" else 0, filter_rule=1 if filt == "nlf" else 0)
        gc, oc = F.Cst(g, ql, qe, cfg), oracle.Cst(o, ql, qe, order=order, filter=filt)
        want = _oracle_bytes(o, oc, ql, qe)
        r = F.match(gc, cfg=cfg)                                   # donation on
        assert r["count"] == want["count"]
        assert F.last_match_floor_bytes() == want["balg"], (order, filt)
        cc = torch.zeros(1, dtype=torch.int64, device="cuda")      # a chunk count: donation off
        r = F.match(gc, cfg=cfg, chunk_counts=cc)
        assert r["count"] == want["count"] == int(cc[0])
        assert F.last_match_floor_bytes() == want["balg"]
        assert want["balg"] <= F.last_match_bytes() <= want["balg_max"]


def test_timed_matcher_floor_under_heavy_donation():
    """A hub under every root run: idle warps take runs all the time; the
    floor counted by the donors and takers together is still the oracle's."""
    rng = np.random.default_rng(13)
    n = 2000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(5000, 2)) if x[0] != x[1]]
    e = np.array(e, np.int32)
    lab = np.zeros(n, np.int32)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    for qe in ([[0, 1], [1, 2], [2, 3]], [[0, 1], [1, 2], [0, 2], [2, 3]]):
        ql = np.zeros(4, np.int32)
        gc, oc = F.Cst(g, ql, qe), oracle.Cst(o, ql, qe)
        want = _oracle_bytes(o, oc, ql, qe)
        for cells in (0, 7):
            r = F.match(gc, cfg=F.default_config(queue_cells=cells))
            assert r["count"] == want["count"]
            assert F.last_match_floor_bytes() == want["balg"], cells


def test_time_budget_reports_timeout():
    n, e, lab = 20_000, synth.chung_lu_edges(20_000, 200_000, 2.1, 5), None
    lab = np.zeros(n, np.int32)
    g = F.Graph(n, e, lab)
    cst = F.Cst(g, np.zeros(6, np.int32), [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]])
    cfg = F.default_config(time_budget_s=0.05)
    r = F.match(cst, cfg=cfg, check=False)
    assert r["status"] == F.FAST_ERR_TIMEOUT
    assert 0 < r["count"] < cst.W


@pytest.mark.parametrize("seed", range(6))
def test_partition_cap_matches_oracle(seed):
    n, e, lab, ql, qe = rand_case(4500 + seed, n_lo=80, n_hi=250, k_hi=6, L_hi=3)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc, oc = F.Cst(g, ql, qe), oracle.Cst(o, ql, qe)
    if gc.W == 0:
        return
    total = oracle.count(o, ql, qe)
    for cap in (1, 3, 10):
        delta = max(1, gc.W // 50)
        ch = F.Chunks(gc, F.default_config(delta_w=delta, max_chunks=cap))
        want = oc.partition(delta, max_chunks=cap)
        assert gpu_chunks_global(gc, ch) == want and ch.n <= cap
        assert F.match(gc, ch)["count"] == total


# ------------------------------------------------------------------- limit

@pytest.mark.parametrize("seed", range(10))
def test_limit_matches_oracle(seed):
    n, e, lab, ql, qe = rand_case(6000 + seed, n_lo=100, n_hi=300, k_hi=5, L_hi=2)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    gc = F.Cst(g, ql, qe)
    total = oracle.count(o, ql, qe)
    for L in (1, 33, max(1, total // 2), total + 1):
        cfg = F.default_config(limit=L)
        kemb = min(L, 1 << 18)                 # rows copied out (the count is always exact)
        r = F.match(gc, k=kemb, cfg=cfg)
        assert r["count"] == min(total, L)
        rows = r["emb"][:r["written"]].astype(np.int32)
        assert r["written"] == min(total, L, kemb)
        assert oracle.invalid_rows(o, ql, qe, rows) == 0
        assert np.unique(rows, axis=0).shape[0] == rows.shape[0]


def test_work_stealing_on_a_skewed_tree():
    """One hub adjacent to everything: almost all work sits under a few root
    runs, so idle warps must take runs from busy ones.  Counts stay exact."""
    rng = np.random.default_rng(11)
    n = 3000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(6000, 2)) if x[0] != x[1]]
    e = np.array(e, np.int32)
    lab = np.zeros(n, np.int32)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    for qe in ([[0, 1], [1, 2], [2, 3]], [[0, 1], [1, 2], [0, 2], [2, 3]]):
        ql = np.zeros(4, np.int32)
        want = oracle.count(o, ql, qe)
        cst = F.Cst(g, ql, qe)
        assert F.match(cst)["count"] == want
        assert F.match(cst, F.Chunks(cst, F.default_config(delta_w=max(1, cst.W // 64))))["count"] == want


@pytest.mark.parametrize("cells", [1, 2, 7, 64])
def test_work_stealing_with_a_tiny_ring(cells):
    """The ring of donated runs wraps around thousands of times and is often
    full (a donor then keeps its work); counts stay exact on every path."""
    rng = np.random.default_rng(12)
    n = 3000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(6000, 2)) if x[0] != x[1]]
    e = np.array(e, np.int32)
    lab = np.zeros(n, np.int32)
    g, o = F.Graph(n, e, lab), oracle.Graph(n, e, lab)
    cfg = F.default_config(queue_cells=cells)
    for qe in ([[0, 1], [1, 2], [2, 3]], [[0, 1], [1, 2], [0, 2], [2, 3]], [[0, 1], [1, 2], [2, 3], [3, 4]]):
        ql = np.zeros(int(np.max(qe)) + 1, np.int32)
        want = oracle.count(o, ql, qe)
        cst = F.Cst(g, ql, qe)
        assert F.match(cst, cfg=cfg)["count"] == want
        assert F.match_noalloc(cst, cfg=cfg)["count"] == want
        lim = F.default_config(queue_cells=cells, limit=max(1, want // 3))
        assert F.match(cst, cfg=lim)["count"] == min(want, max(1, want // 3))
    qs = [(np.zeros(4, np.int32), [[0, 1], [1, 2], [2, 3]]), (np.zeros(4, np.int32), [[0, 1], [1, 2], [0, 2], [2, 3]])]
    counts, status = F.Batch(g, 4, cfg).run(qs * 2)
    assert status.tolist() == [0] * 4
    assert counts.tolist() == [oracle.count(o, ql, qe) for ql, qe in qs] * 2


# ------------------------------------------------- power-law graph, full size

@pytest.fixture(scope="module")
def powerlaw():
    n, e, lab = synth.powerlaw_graph()          # 1M vertices, 16M edges, 16 Zipf labels
    qs = []
    for k in (8, 16):
        for kind in ("dense", "sparse"):
            qs += synth.walk_queries(n, e, lab, k, 1, kind, seed=2000, stream0=1000 * k + (0 if kind == "dense" else 500))
    return n, e, lab, qs, F.Graph(n, e, lab), oracle.Graph(n, e, lab)


def test_powerlaw_loader(powerlaw):
    n, e, lab, qs, g, o = powerlaw
    goff, gcol = g.csr()
    ooff, ocol = csr_by_label(*o.csr(), lab)
    assert np.array_equal(goff, ooff) and np.array_equal(gcol, ocol)


def test_powerlaw_cst(powerlaw):
    n, e, lab, qs, g, o = powerlaw
    q = qs[0]
    compare_cst(F.Cst(g, q.labels, q.edges), oracle.Cst(o, q.labels, q.edges), q.k)


@pytest.mark.parametrize("qi", range(4))
def test_powerlaw_limit_counts_and_embeddings(powerlaw, qi):
    """min(total, L) at full size, against the oracle's own search; every
    embedding written is checked against Definition 1 and is distinct."""
    n, e, lab, qs, g, o = powerlaw
    q = qs[qi]
    L = 1 << 18
    cfg = F.default_config(limit=L, delta_w=1 << 20, max_chunks=4096, time_budget_s=60.0)
    cst = F.Cst(g, q.labels, q.edges, cfg)
    ch = F.Chunks(cst, cfg)
    r = F.match(cst, ch, k=L, cfg=cfg)
    want = oracle.match(o, q.labels, q.edges, limit=L)
    assert want["complete"]
    assert r["count"] == want["count"]
    rows = r["emb"][:r["written"]].astype(np.int32)
    assert rows.shape[0] == min(L, r["count"])
    assert oracle.invalid_rows(o, q.labels, q.edges, rows) == 0
    assert len(set(map(tuple, rows.tolist()))) == rows.shape[0]
