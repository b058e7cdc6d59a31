"""Pins for the oracle: checks against what the paper and the mathematics fix
(brute force, closed forms, automorphism and order invariants, the soundness
theorem of Sec. IV-A, and the worked examples of Sec. IV-B, IV-C and V-A).
CPU only."""
import itertools
import json
import math
import os

import networkx as nx
import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers

def random_graph(rng, n, p, L):
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    labels = rng.integers(0, L, size=n).astype(np.int32)
    return np.array(edges, dtype=np.int32).reshape(-1, 2), labels


def random_connected_query(rng, k, L, extra_p):
    edges = set()
    for v in range(1, k):
        edges.add((int(rng.integers(0, v)), v))
    for a in range(k):
        for b in range(a + 1, k):
            if rng.random() < extra_p:
                edges.add((a, b))
    labels = rng.integers(0, L, size=k).astype(np.int32)
    return labels, np.array(sorted(edges), dtype=np.int32).reshape(-1, 2)


def relabel_query(labels, edges, perm):
    """query vertex u becomes perm[u]"""
    nl = np.empty_like(labels)
    nl[perm] = labels
    ne = np.array([[perm[a], perm[b]] for a, b in edges], dtype=np.int32).reshape(-1, 2)
    return nl, ne


def aut_count(labels, edges):
    k = len(labels)
    E = {(min(a, b), max(a, b)) for a, b in edges}
    n = 0
    for p in itertools.permutations(range(k)):
        if all(labels[p[u]] == labels[u] for u in range(k)) and \
           all((min(p[a], p[b]), max(p[a], p[b])) in E for a, b in E):
            n += 1
    return n


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("seed", range(60))
def test_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    k = int(rng.integers(1, min(5, n) + 1))
    L = int(rng.integers(1, 4))
    edges, labels = random_graph(rng, n, float(rng.uniform(0.25, 0.8)), L)
    ql, qe = random_connected_query(rng, k, L, float(rng.uniform(0.0, 0.6)))
    want = oracle.brute_force(n, edges, labels, ql, qe)
    g = oracle.Graph(n, edges, labels)
    r = oracle.match(g, ql, qe, max_emb=100000, threads=1)
    assert r["complete"]
    assert r["count"] == len(want)
    got = [tuple(int(x) for x in row) for row in r["emb"]]
    assert got == want


def test_duplicates_and_loops_are_dropped():
    # the paper's graphs are simple (Sec. II-A): repeats and loops carry no edge
    edges = np.array([[0, 1], [1, 0], [0, 1], [1, 1], [1, 2], [2, 2]], np.int32)
    g = oracle.Graph(3, edges, np.zeros(3, np.int32))
    off, adj = g.csr()
    assert off.tolist() == [0, 1, 3, 4]
    assert adj.tolist() == [1, 0, 2, 1]
    assert oracle.count(g, [0, 0], [[0, 1]]) == 4   # 2 edges, both directions


# ----------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,k", [(5, 1), (5, 2), (5, 3), (6, 4), (7, 5), (8, 3)])
def test_clique_in_complete_graph(n, k):
    edges = np.array(list(itertools.combinations(range(n), 2)), np.int32)
    g = oracle.Graph(n, edges, np.zeros(n, np.int32))
    qe = np.array(list(itertools.combinations(range(k), 2)), np.int32).reshape(-1, 2)
    assert oracle.count(g, np.zeros(k, np.int32), qe) == math.perm(n, k)


@pytest.mark.parametrize("n,L", [(3, 1), (5, 2), (6, 5), (9, 4), (12, 11), (40, 7)])
def test_path_in_cycle(n, L):
    edges = np.array([[i, (i + 1) % n] for i in range(n)], np.int32)
    g = oracle.Graph(n, edges, np.zeros(n, np.int32))
    qe = np.array([[i, i + 1] for i in range(L)], np.int32)
    assert oracle.count(g, np.zeros(L + 1, np.int32), qe) == 2 * n


@pytest.mark.parametrize("seed", range(6))
def test_star_counts(seed):
    rng = np.random.default_rng(100 + seed)
    n = 60
    edges, labels = random_graph(rng, n, 0.15, 3)
    g = oracle.Graph(n, edges, labels)
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b); adj[b].add(a)
    for s in (1, 2, 3):
        for a_lab in range(3):
            for b_lab in range(3):
                want = sum(math.perm(sum(1 for w in adj[v] if labels[w] == b_lab), s)
                           for v in range(n) if labels[v] == a_lab)
                ql = np.array([a_lab] + [b_lab] * s, np.int32)
                qe = np.array([[0, i] for i in range(1, s + 1)], np.int32)
                assert oracle.count(g, ql, qe) == want


def test_single_edge_counts():
    rng = np.random.default_rng(7)
    n = 80
    edges, labels = random_graph(rng, n, 0.1, 3)
    g = oracle.Graph(n, edges, labels)
    for a in range(3):
        for b in range(3):
            m_ab = sum(1 for x, y in edges if {labels[x], labels[y]} == {a, b})
            want = m_ab * (2 if a == b else 1)
            assert oracle.count(g, [a, b], [[0, 1]]) == want


@pytest.mark.parametrize("seed", range(4))
def test_triangles_against_networkx(seed):
    rng = np.random.default_rng(200 + seed)
    n = 70
    edges, labels = random_graph(rng, n, 0.12, 1)
    G = nx.Graph(); G.add_nodes_from(range(n)); G.add_edges_from(edges.tolist())
    tri = sum(nx.triangles(G).values()) // 3
    g = oracle.Graph(n, edges, labels)
    assert oracle.count(g, [0, 0, 0], [[0, 1], [1, 2], [0, 2]]) == 6 * tri


# -------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(10))
def test_embeddings_equal_copies_times_automorphisms(seed):
    rng = np.random.default_rng(300 + seed)
    n = 9
    edges, labels = random_graph(rng, n, 0.5, 2)
    k = int(rng.integers(2, 5))
    ql, qe = random_connected_query(rng, k, 2, 0.5)
    g = oracle.Graph(n, edges, labels)
    r = oracle.match(g, ql, qe, max_emb=1 << 16)
    copies = set()
    for M in r["emb"].tolist():
        copies.add(frozenset((min(M[a], M[b]), max(M[a], M[b])) for a, b in qe) | frozenset((v,) for v in M))
    assert r["count"] == len(copies) * aut_count(ql, qe)


@pytest.mark.parametrize("seed", range(8))
def test_count_independent_of_order_and_vertex_ids(seed):
    rng = np.random.default_rng(400 + seed)
    n = 40
    edges, labels = random_graph(rng, n, 0.15, 2)
    k = 5
    ql, qe = random_connected_query(rng, k, 2, 0.3)
    g = oracle.Graph(n, edges, labels)
    base = oracle.match(g, ql, qe, max_emb=1 << 18)
    # another connected order: BFS from a different query vertex
    qperm = rng.permutation(k)
    ql2, qe2 = relabel_query(ql, qe, qperm)
    r2 = oracle.match(g, ql2, qe2, max_emb=1 << 18)
    assert r2["count"] == base["count"]
    back = r2["emb"][:, qperm] if r2["count"] else r2["emb"]
    assert sorted(map(tuple, back.tolist())) == sorted(map(tuple, base["emb"].tolist()))
    # relabelling G's vertices permutes the embedding set
    gp = rng.permutation(n)
    g3 = oracle.Graph(n, gp[edges], labels[np.argsort(gp)])
    r3 = oracle.match(g3, ql, qe, max_emb=1 << 18)
    assert r3["count"] == base["count"]
    inv = np.argsort(gp)
    mapped = sorted(map(tuple, inv[r3["emb"]].tolist())) if r3["count"] else []
    assert mapped == sorted(map(tuple, base["emb"].tolist()))


# ------------------------------------------------------ CST (Algorithm 1)

def _cst_case(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(30, 120))
    edges, labels = random_graph(rng, n, float(rng.uniform(0.05, 0.25)), int(rng.integers(1, 4)))
    k = int(rng.integers(2, 7))
    ql, qe = random_connected_query(rng, k, int(labels.max()) + 1, float(rng.uniform(0, 0.4)))
    return n, edges, labels, ql, qe


@pytest.mark.parametrize("seed", range(25))
def test_cst_is_sound(seed):
    """Soundness (Sec. IV-A): every embedding maps u into C(u), and every
    query edge onto a CST edge; so the CST is a complete search space."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    r = oracle.match(g, ql, qe, max_emb=1 << 18)
    k = len(ql)
    cand = [set(c.cand(u).tolist()) for u in range(k)]
    tree = {}
    for u in range(k):
        if c.parent[u] >= 0:
            off, vals = c.tree(u)
            cp = c.cand(int(c.parent[u]))
            tree[u] = {int(cp[i]): set(vals[off[i]:off[i + 1]].tolist()) for i in range(len(cp))}
    nts = {(a, b): (off, vals, c.cand(a)) for a, b, off, vals in c.nontree()}
    for M in r["emb"].tolist():
        for u in range(k):
            assert M[u] in cand[u]
            if c.parent[u] >= 0:
                assert M[u] in tree[u][M[int(c.parent[u])]]
        for (a, b), (off, vals, ca) in nts.items():
            i = int(np.searchsorted(ca, M[a]))
            assert M[b] in set(vals[off[i]:off[i + 1]].tolist())
    # the tree's own counts: W bounds the embedding count (Sec. IV-C)
    wf, wi, _, _ = c.workload()
    assert wi >= r["count"] and wf >= r["count"]


@pytest.mark.parametrize("seed", range(25))
def test_cst_lists_follow_definition(seed):
    """Each list is N_G(v) restricted to the other end's candidate set (the
    CST definition of Sec. IV-A), candidates carry the query label, and every
    candidate has its children (bottom-up validity)."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    off_g, adj_g = g.csr()
    N = lambda v: set(adj_g[off_g[v]:off_g[v + 1]].tolist())
    k = len(ql)
    dq = np.bincount(qe.ravel(), minlength=k)
    for u in range(k):
        for v in c.cand(u).tolist():
            assert labels[v] == ql[u] and len(N(v)) >= dq[u]
    children = {u: [w for w in range(k) if c.parent[w] == u] for u in range(k)}
    for u in range(k):
        if c.parent[u] < 0:
            continue
        off, vals = c.tree(u)
        cp, cu = c.cand(int(c.parent[u])), set(c.cand(u).tolist())
        for i, vp in enumerate(cp.tolist()):
            assert vals[off[i]:off[i + 1]].tolist() == sorted(N(vp) & cu)
    for u in range(k):
        for w in children[u]:
            off, vals = c.tree(w)
            assert np.all(np.diff(off) > 0)       # every survivor keeps each child
    for a, b, off, vals in c.nontree():
        cb = set(c.cand(b).tolist())
        for i, v in enumerate(c.cand(a).tolist()):
            assert vals[off[i]:off[i + 1]].tolist() == sorted(N(v) & cb)


@pytest.mark.parametrize("seed", range(12))
def test_workload_equals_count_for_trees_with_distinct_labels(seed):
    """W ignores injectivity and non-tree edges (Sec. IV-C); for a tree query
    whose labels are pairwise distinct neither matters, so W is exact."""
    rng = np.random.default_rng(600 + seed)
    n = 150
    L = 6
    edges, labels = random_graph(rng, n, 0.06, L)
    k = int(rng.integers(2, 6))
    ql = rng.permutation(L)[:k].astype(np.int32)
    qe = np.array([[int(rng.integers(0, v)), v] for v in range(1, k)], np.int32)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    wf, wi, _, _ = c.workload()
    cnt = oracle.count(g, ql, qe)
    assert wi == cnt and wf == float(cnt)


# ------------------------------------------------------- paper's examples

def _fixture():
    with open(os.path.join(GOLDEN, "paper_fig4_example.json")) as f:
        return json.load(f)


def test_paper_workload_example():
    fx = _fixture()
    g = oracle.Graph(fx["n"], fx["edges"], fx["labels"])
    c = oracle.Cst(g, fx["query_labels"], fx["query_edges"])
    ex = fx["expected"]
    assert c.root == ex["root"]
    assert c.parent.tolist() == ex["tree_parent"]
    wf, wi, cf, ci = c.workload(dump_u=0)
    assert wi == ex["W"] and wf == ex["W"]
    cand0 = c.cand(0).tolist()
    for v, want in ex["c_u0"].items():
        assert int(ci[cand0.index(int(v))]) == want


def test_paper_partition_example():
    fx = _fixture()
    ex = fx["expected"]
    g = oracle.Graph(fx["n"], fx["edges"], fx["labels"])
    c = oracle.Cst(g, fx["query_labels"], fx["query_edges"])
    chunks = c.partition(ex["partition_delta_w"])
    assert [(a, b, w) for (j, pre, a, b, w, i) in chunks] == [tuple(x) for x in ex["partition_chunks"]]
    # parts are disjoint and complete: their counts add up to the whole
    total = oracle.count(g, fx["query_labels"], fx["query_edges"])
    parts = [oracle.count(g, fx["query_labels"], fx["query_edges"], allow=c.chunk_allow(j, pre, a, b))
             for (j, pre, a, b, w, i) in chunks]
    assert sum(parts) == total


def test_paper_generator_validator_round():
    fx = _fixture()
    ex = fx["expected"]
    g = oracle.Graph(fx["n"], fx["edges"], fx["labels"])
    ql = np.array(fx["query_labels"], np.int32)
    qe = np.array(fx["query_edges"], np.int32)
    # partial results over (u0, u1), root fixed to v1: the round's input P
    r2 = oracle.match(g, ql[:2], [[0, 1]], allow={0: [1]}, max_emb=100)
    assert r2["emb"].tolist() == ex["round_P"]
    # one more position, u2, with its tree edge (u0,u2) and non-tree edge (u1,u2)
    sub_e = [[a, b] for a, b in qe.tolist() if a < 3 and b < 3]
    r3 = oracle.match(g, ql[:3], sub_e, order=[0, 1, 2], allow={0: [1]}, max_emb=100)
    assert r3["emb"].tolist() == ex["round_survivors"]
    gen = ex["round_generated"]
    bn = [1 if row in ex["round_survivors"] else 0 for row in gen]
    assert bn == ex["round_B_n"]
    # the order of the example reaches the same embeddings as any other
    full = oracle.match(g, ql, qe, max_emb=100)
    alt = oracle.match(g, ql, qe, order=ex["round_order"], max_emb=100)
    assert full["emb"].tolist() == alt["emb"].tolist() and full["count"] == 3


# ------------------------------------------------------------- partition

@pytest.mark.parametrize("seed", range(10))
def test_partition_disjoint_and_complete(seed):
    n, edges, labels, ql, qe = _cst_case(700 + seed)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    wf, wi, _, _ = c.workload()
    total = oracle.match(g, ql, qe, max_emb=1 << 18)
    delta = max(1, wi // 7)
    chunks = c.partition(delta)
    seen = set()
    s = 0
    for (j, pre, a, b, w, i) in chunks:
        assert 0 < w <= delta or (b - a == 1 and j == len(ql) - 1)
        assert c.chunk_w(j, pre, c.chunk_list(j, pre)[a:b]) == w
        r = oracle.match(g, ql, qe, allow=c.chunk_allow(j, pre, a, b), max_emb=1 << 18)
        assert r["count"] <= w
        rows = set(map(tuple, r["emb"].tolist()))
        assert len(rows) == min(r["count"], 1 << 18) and not (rows & seen)
        seen |= rows
        s += r["count"]
    assert s == total["count"]
    if total["count"] <= 1 << 18:
        assert seen == set(map(tuple, total["emb"].tolist()))


def test_partition_sampling_keeps_a_subset():
    n, edges, labels, ql, qe = _cst_case(801)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    wf, wi, _, _ = c.workload()
    full = c.partition(max(1, wi // 20))
    samp = c.partition(max(1, wi // 20), c_root=2.0, c_deep=1.0, seed=5)
    ids = {ch[-1] for ch in full}
    assert len(samp) <= len(full) and all(ch[-1] in ids for ch in samp)


# ------------------------------------------------------ algorithmic bytes

def test_balg_counts_lists_of_extended_partials():
    """The byte count of the enumerator, on a path a-b-c where every list
    is known by hand."""
    # 0(a)-1(b)-2(c), 0-3(b), 3-4(c), 3-5(c)
    edges = [[0, 1], [1, 2], [0, 3], [3, 4], [3, 5]]
    labels = [0, 1, 2, 1, 2, 2]
    g = oracle.Graph(6, edges, labels)
    r = oracle.match(g, [0, 1, 2], [[0, 1], [1, 2]], want_balg=True, want_depth=True)
    assert r["count"] == 3
    # extend {0}: image 4 + offsets 16 + list {1,3} 2*4; extend {0,1}: 4 + 16 + {2} 4;
    # extend {0,3}: 4 + 16 + {4,5} 2*4
    assert r["balg"] == (4 + 16 + 8) + (4 + 16 + 4) + (4 + 16 + 8)
    assert r["depth"].tolist() == [1, 2, 3]


def test_balg_floor_and_ceiling_on_a_triangle_query():
    """A triangle query: one non-tree list per extension at the last
    position; floor and ceiling by hand."""
    # star centre 0 (a) with leaves 1..4 (b); leaves 1-2 and 3-4 joined
    edges = [[0, 1], [0, 2], [0, 3], [0, 4], [1, 2], [3, 4]]
    labels = [0, 1, 1, 1, 1]
    g = oracle.Graph(5, edges, labels)
    # q: a-b, a-b', b-b' in order (0, 1, 2), parents (-, 0, 0)
    r = oracle.match(g, [0, 1, 1], [[0, 1], [0, 2], [1, 2]], order=[0, 1, 2], par=[0, 0, 0],
                     want_balg=True, want_depth=True)
    assert r["count"] == 4 and r["depth"].tolist() == [1, 4, 4]
    # extend {0}: image 4 + tree offsets 16 + tree list {1,2,3,4} 16 = 36
    # extend {0,x}, x a leaf: image 4 + two lists' offsets 32; the generator is
    #   the shorter non-tree list {x's twin} (1 entry, 4 B) rather than the
    #   4-entry tree list; that entry is in both lists and position 1 has its
    #   label: its data vertex 4
    floor = 36 + 4 * (4 + 32 + 4 + 4)
    assert r["balg"] == floor
    # ceiling per extension {0,x}: the other list (the tree list, 4 entries)
    #   merged against one segment: 4 (4 + 32) tile bytes plus one gallop of
    #   six 32-probe rounds, 4 * 32 * 6
    assert r["balg_max"] == floor + 4 * (4 * (4 + 32) + 4 * 32 * 6)


def _brute_balg(n, edges, labels, ql, qe, order, par, cand):
    """The floor and ceiling of the extension bytes by brute force: every
    injective map of the first d positions (d = 1 .. k-1) that keeps labels,
    candidate sets and every query edge among them is a valid partial, and
    is extended once; its lists are the CST lists by definition (the
    neighbours of an image that lie in the next position's candidate set)."""
    k = len(ql)
    adj = [set() for _ in range(n)]
    for a, b in np.asarray(edges).reshape(-1, 2).tolist():
        if a != b:
            adj[a].add(b); adj[b].add(a)
    A = set()
    for a, b in np.asarray(qe).reshape(-1, 2).tolist():
        A.add((a, b)); A.add((b, a))
    lo = hi = 0.0
    for d in range(1, k):
        us = [int(order[i]) for i in range(d)]
        u = int(order[d])
        back = [i for i in range(d) if (us[i], u) in A and i != par[d]]
        same = any(ql[x] == ql[u] for x in us)
        for M in itertools.permutations(range(n), d):
            if any(M[i] not in cand[us[i]] for i in range(d)):
                continue
            if any((us[i], us[j]) in A and M[j] not in adj[M[i]] for i in range(d) for j in range(i)):
                continue
            lists = [sorted(w for w in adj[M[i]] if w in cand[u]) for i in [par[d]] + back]
            gi = min(range(len(lists)), key=lambda j: (len(lists[j]), j))
            G = lists[gi]
            inter = sum(all(x in L for L in lists) for x in G)
            f = 4 + 16 * len(lists) + 4 * len(G) + (4 * inter if same else 0)
            segs = (len(G) + 31) // 32
            extra = 0
            if G:
                for j, L in enumerate(lists):
                    if j != gi:
                        extra += 4 * (len(L) + 32 * segs) + 4 * 32 * 6 * min(len(G), (len(L) + 31) // 32 + segs)
            lo += f
            hi += f + extra
    return lo, hi


@pytest.mark.parametrize("seed", range(10))
def test_balg_floor_and_ceiling_by_brute_force(seed):
    """The oracle's byte floor and ceiling equal a brute-force sum over every
    valid partial embedding of every prefix of the matching order, both
    orders, on tiny random cases (allowed sets = the CST's candidate sets)."""
    rng = np.random.default_rng(7300 + seed)
    n = int(rng.integers(7, 10))
    edges, labels = random_graph(rng, n, float(rng.uniform(0.3, 0.7)), int(rng.integers(1, 3)))
    k = int(rng.integers(3, 5))
    ql, qe = random_connected_query(rng, k, int(labels.max()) + 1, 0.6)
    g = oracle.Graph(n, edges, labels)
    for order_rule in ("path", "greedy"):
        c = oracle.Cst(g, ql, qe, order=order_rule)
        cand = [set(c.cand(u).tolist()) for u in range(k)]
        par = _tree_par(c)
        r = oracle.match(g, ql, qe, order=c.order, par=par, allow={u: cand[u] for u in range(k)}, want_balg=True)
        lo, hi = _brute_balg(n, edges, labels, ql, qe, [int(x) for x in c.order], par, cand)
        assert r["balg"] == lo and r["balg_max"] == hi, (order_rule, r["balg"], lo, r["balg_max"], hi)


# ------------------------------------------------------------------- limit

@pytest.mark.parametrize("seed", range(8))
def test_limit_gives_min_of_total_and_limit(seed):
    rng = np.random.default_rng(900 + seed)
    n = 60
    edges, labels = random_graph(rng, n, 0.2, 2)
    ql, qe = random_connected_query(rng, 4, 2, 0.3)
    g = oracle.Graph(n, edges, labels)
    full = oracle.match(g, ql, qe, max_emb=1 << 20)
    allrows = set(map(tuple, full["emb"].tolist()))
    for L in (1, 7, max(1, full["count"] // 3), full["count"], full["count"] + 5):
        r = oracle.match(g, ql, qe, limit=L, max_emb=1 << 20)
        assert r["complete"] and r["count"] == min(full["count"], L)
        rows = set(map(tuple, r["emb"].tolist()))
        assert len(rows) == r["count"] and rows <= allrows


def test_embedding_checker_rejects_each_kind_of_fault():
    g = oracle.Graph(4, [[0, 1], [1, 2], [2, 3]], [0, 1, 0, 1])
    ql, qe = [0, 1, 0], [[0, 1], [1, 2]]
    assert oracle.invalid_rows(g, ql, qe, [[0, 1, 2], [2, 1, 0], [2, 3, 2]]) == 1   # repeat
    assert oracle.invalid_rows(g, ql, qe, [[0, 3, 2]]) == 1                          # missing edge
    assert oracle.invalid_rows(g, ql, qe, [[1, 0, 2]]) == 1                          # labels
    assert oracle.invalid_rows(g, ql, qe, [[0, 1, 2]]) == 0


@pytest.mark.parametrize("seed", range(6))
def test_partition_cap_keeps_chunks_disjoint_and_complete(seed):
    n, edges, labels, ql, qe = _cst_case(950 + seed)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe)
    wf, wi, _, _ = c.workload()
    if wi == 0:
        return
    total = oracle.count(g, ql, qe)
    nroot = len(c.cand(c.root))
    for cap in (1, 3, 10):
        dw = max(1, wi // 50)
        chunks = c.partition(dw, max_chunks=cap)
        assert len(chunks) <= cap
        s = sum(oracle.count(g, ql, qe, allow=c.chunk_allow(j, pre, a, b)) for (j, pre, a, b, w, i) in chunks)
        assert s == total
        # a root split wider than the cap is cut to exactly `cap` runs of the root list
        if min(-(-wi // dw), nroot) > cap:
            assert len(chunks) == cap
            assert all(j == 0 for (j, pre, a, b, w, i) in chunks)
            assert sorted((a, b) for (j, pre, a, b, w, i) in chunks)[0][0] == 0


# ------------------------------------------------- matching order (greedy)

def _tree_par(c):
    """Per position of c.order, the position of its t_q parent (0 at the root)."""
    pos = {int(u): i for i, u in enumerate(c.order)}
    return [pos[int(c.parent[int(u)])] if c.parent[int(u)] >= 0 else 0 for u in c.order]


def test_greedy_order_house_in_k6():
    """Hand-worked: the 'house' query (square 0-1-2-3 plus roof 4 on 0 and
    1) in K6.  Every C0 is all six vertices, so the root is 0 (ties with 1
    at 6/3, smaller id) and t_q is 0 -> {1, 3, 4}, 1 -> {2}.  Path-based:
    0, then its children by (|C|, id) with 1's subtree first: 0 1 2 3 4.
    Greedy: after 0 the frontier 1, 3, 4 has one edge each (1 by id); then
    4 has two edges to {0, 1} against one for 2 and 3; then 2 before 3 by
    id: 0 1 4 2 3.  Either order finds 6!/1! = 720 embeddings."""
    n = 6
    edges = [[a, b] for a in range(n) for b in range(a + 1, n)]
    g = oracle.Graph(n, edges, [0] * n)
    ql, qe = [0] * 5, [[0, 1], [1, 2], [2, 3], [3, 0], [0, 4], [1, 4]]
    path = oracle.Cst(g, ql, qe)
    greedy = oracle.Cst(g, ql, qe, order="greedy")
    assert path.root == greedy.root == 0
    assert path.parent.tolist() == greedy.parent.tolist() == [-1, 0, 1, 0, 0]
    assert path.order.tolist() == [0, 1, 2, 3, 4]
    assert greedy.order.tolist() == [0, 1, 4, 2, 3]
    for c in (path, greedy):
        assert oracle.count(g, ql, qe, order=c.order.tolist(), par=_tree_par(c)) == 720


def test_bfs_and_fewest_candidate_orders_house_in_k6():
    """Hand-worked, the house in K6 again (t_q: 0 -> {1, 3, 4}, 1 -> {2}).
    BFS order (rule 2): the order t_q was built in, 0 1 3 4 2.  Fewest
    candidates first (rule 3): every |C| is 6, so ties go by id along the
    frontier: 0, then 1 (of 1, 3, 4), then 2 (of 2, 3, 4), then 3, 4."""
    n = 6
    edges = [[a, b] for a in range(n) for b in range(a + 1, n)]
    g = oracle.Graph(n, edges, [0] * n)
    ql, qe = [0] * 5, [[0, 1], [1, 2], [2, 3], [3, 0], [0, 4], [1, 4]]
    bfs = oracle.Cst(g, ql, qe, order="bfs")
    few = oracle.Cst(g, ql, qe, order="mincand")
    assert bfs.order.tolist() == [0, 1, 3, 4, 2] == bfs.bfs.tolist()
    assert few.order.tolist() == [0, 1, 2, 3, 4]
    for c in (bfs, few):
        assert oracle.count(g, ql, qe, order=c.order.tolist(), par=_tree_par(c)) == 720


def test_fewest_candidates_against_greedy_by_hand():
    """A labelled case where the rules part: q0 (label 0) joined to q1, q2,
    q3 (labels 1, 2, 3) and q1-q2.  G: vertex 0 (label 0) joined to 1
    (label 1), to 3..7 (label 2) and to 8..10 (label 3); vertex 1 joined to
    3..7.  |C| = 1, 1, 5, 3; the root is q0 (1/3 below 1/2) and t_q is the
    star q0 -> q1, q2, q3.  Greedy (rule 1): q1 (fewest candidates among one
    edge each), then q2 (two edges to placed vertices), then q3: 0 1 2 3.
    Fewest candidates (rule 3): q1, then q3 (3 < 5), then q2: 0 1 3 2, which
    is also the path-based order (children by |C|).  BFS: 0 1 2 3.  Every
    order finds 1 x 1 x 5 x 3 = 15 embeddings."""
    labels = [0, 1] + [9] + [2] * 5 + [3] * 3
    edges = [[0, 1]] + [[0, v] for v in range(3, 8)] + [[0, v] for v in range(8, 11)] + [[1, v] for v in range(3, 8)]
    g = oracle.Graph(11, edges, labels)
    ql, qe = [0, 1, 2, 3], [[0, 1], [0, 2], [0, 3], [1, 2]]
    want = {"path": [0, 1, 3, 2], "greedy": [0, 1, 2, 3], "bfs": [0, 1, 2, 3], "mincand": [0, 1, 3, 2]}
    for rule, order in want.items():
        c = oracle.Cst(g, ql, qe, order=rule)
        assert c.root == 0 and c.parent.tolist() == [-1, 0, 0, 0]
        assert [len(c.cand(u)) for u in range(4)] == [1, 1, 5, 3]
        assert c.order.tolist() == order, rule
        assert oracle.count(g, ql, qe, order=c.order.tolist(), par=_tree_par(c)) == 15


@pytest.mark.parametrize("seed", range(25))
def test_all_order_rules_connected_and_count_invariant(seed):
    """Every rule places each vertex after its t_q parent, rule 2 is exactly
    the BFS order, and matching in any of the four orders finds the same
    number of embeddings."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    want = oracle.count(g, ql, qe)
    k = len(ql)
    for rule in ("bfs", "mincand"):
        c = oracle.Cst(g, ql, qe, order=rule)
        pos = {int(u): i for i, u in enumerate(c.order)}
        assert sorted(pos) == list(range(k)) and int(c.order[0]) == c.root
        for u in range(k):
            if c.parent[u] >= 0:
                assert pos[int(c.parent[u])] < pos[u]
        if rule == "bfs":
            assert c.order.tolist() == c.bfs.tolist()
        assert oracle.count(g, ql, qe, order=c.order.tolist(), par=_tree_par(c)) == want


@pytest.mark.parametrize("seed", range(25))
def test_greedy_order_is_connected_and_count_invariant(seed):
    """Every vertex follows its t_q parent (so the CST's tree lists apply);
    matching in the greedy order finds the same embeddings, and the CST is
    the same one but for the direction of the non-tree lists."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    path = oracle.Cst(g, ql, qe)
    greedy = oracle.Cst(g, ql, qe, order="greedy")
    k = len(ql)
    pos = {int(u): i for i, u in enumerate(greedy.order)}
    assert sorted(pos) == list(range(k)) and int(greedy.order[0]) == greedy.root
    for u in range(k):
        if greedy.parent[u] >= 0:
            assert pos[int(greedy.parent[u])] < pos[u]
    for u in range(k):
        assert np.array_equal(path.cand(u), greedy.cand(u))
    want = oracle.count(g, ql, qe)
    assert oracle.count(g, ql, qe, order=greedy.order.tolist(), par=_tree_par(greedy)) == want
    assert greedy.workload()[1] == path.workload()[1]


# --------------------------------------- candidate filter: label frequencies

def test_nlf_filter_hand_case():
    """Query: centre u0 (label 0) joined to u1, u2 (label 1).  Data vertex 0
    (label 0) has neighbours 1 (label 1) and 2 (label 2); vertex 3 (label 0)
    has neighbours 4, 5 (label 1).  The degree filter keeps 0 and 3 for u0;
    the label-frequency filter needs two neighbours labelled 1 and keeps only
    3.  Either way there are 2 embeddings (u1, u2 onto 4, 5 in both orders)."""
    g = oracle.Graph(6, [[0, 1], [0, 2], [3, 4], [3, 5]], [0, 1, 2, 0, 1, 1])
    ql, qe = [0, 1, 1], [[0, 1], [0, 2]]
    ldf = oracle.Cst(g, ql, qe)
    nlf = oracle.Cst(g, ql, qe, filter="nlf")
    assert ldf.c0_count.tolist() == [2, 3, 3]
    assert nlf.c0_count.tolist() == [1, 3, 3]
    assert nlf.cand(0).tolist() == [3]
    assert 0 in ldf.cand(0).tolist()
    assert oracle.count(g, ql, qe) == 2


@pytest.mark.parametrize("seed", range(25))
def test_nlf_filter_is_sound_and_stronger(seed):
    """Every embedding maps u into the label-frequency CST's C(u), and each
    of its candidate sets lies inside the degree filter's."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    ldf = oracle.Cst(g, ql, qe)
    nlf = oracle.Cst(g, ql, qe, filter="nlf")
    k = len(ql)
    r = oracle.match(g, ql, qe, max_emb=1 << 18)
    cand = [set(nlf.cand(u).tolist()) for u in range(k)]
    for row in r["emb"].tolist():
        for u in range(k):
            assert row[u] in cand[u]
    assert all(a <= b for a, b in zip(nlf.c0_count.tolist(), ldf.c0_count.tolist()))
    for u in range(k):
        # with the same root (so the same t_q) the refined sets shrink too
        assert set(nlf.cand(u).tolist()) <= set(ldf.cand(u).tolist()) or nlf.root != ldf.root


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("order,filt", [("greedy", "ldf"), ("path", "nlf"), ("greedy", "nlf")])
def test_partition_complete_for_every_order_and_filter(seed, order, filt):
    """Alg. 2 over the CST of either matching order and either candidate
    filter: the chunks' counts add up to the embeddings of the plain
    definition (disjoint and complete), with and without the chunk cap."""
    n, edges, labels, ql, qe = _cst_case(930 + seed)
    g = oracle.Graph(n, edges, labels)
    c = oracle.Cst(g, ql, qe, order=order, filter=filt)
    wf, wi, _, _ = c.workload()
    total = oracle.count(g, ql, qe)
    if wi == 0:
        assert total == 0
        return
    for cap in (1 << 16, 5):
        chunks = c.partition(max(1, wi // 30), max_chunks=cap)
        s = sum(oracle.count(g, ql, qe, allow=c.chunk_allow(j, pre, a, b)) for (j, pre, a, b, w, i) in chunks)
        assert s == total


# ------------------------------------------------- fixpoint refinement

def test_fixpoint_refinement_hand_case():
    """One bottom-up pass, as the paper writes it, keeps the B candidates of a
    parent candidate that is removed after them; the fixpoint removes them.
    Query A-B, A-C rooted at A; in G, a2 has two B neighbours and no C
    neighbour."""
    e = np.array([(0, 1), (0, 2), (3, 4), (3, 5)], np.int32)
    lab = np.array([0, 1, 2, 0, 1, 1], np.int32)
    g = oracle.Graph(6, e, lab)
    ql, qe = np.array([0, 1, 2], np.int32), np.array([(0, 1), (0, 2)], np.int32)
    once, fix = oracle.Cst(g, ql, qe), oracle.Cst(g, ql, qe, refine="fixpoint")
    assert once.root == fix.root == 0
    assert [once.cand(u).tolist() for u in range(3)] == [[0], [1, 4, 5], [2]]
    assert [fix.cand(u).tolist() for u in range(3)] == [[0], [1], [2]]
    assert once.workload()[1] == fix.workload()[1] == oracle.count(g, ql, qe) == 1


@pytest.mark.parametrize("seed", range(25))
def test_fixpoint_refinement_is_sound_tighter_and_arc_consistent(seed):
    """The fixpoint keeps every embedding's images, lies inside the single
    pass's sets (same root and t_q), and is arc consistent: along every query
    edge, tree or not, each candidate has a neighbour among the other end's
    candidates.  W can only drop and still bounds the count."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    once = oracle.Cst(g, ql, qe)
    fix = oracle.Cst(g, ql, qe, refine="fixpoint")
    k = len(ql)
    off_g, adj_g = g.csr()
    N = lambda v: set(adj_g[off_g[v]:off_g[v + 1]].tolist())
    C = [set(fix.cand(u).tolist()) for u in range(k)]
    assert fix.root == once.root and fix.parent.tolist() == once.parent.tolist()
    for u in range(k):
        assert C[u] <= set(once.cand(u).tolist())
    r = oracle.match(g, ql, qe, max_emb=1 << 18)
    for row in r["emb"].tolist():
        for u in range(k):
            assert row[u] in C[u]
    for a, b in qe.tolist():
        for x, y in ((a, b), (b, a)):
            for v in C[x]:
                assert N(v) & C[y], (x, y, v)
    assert r["count"] <= fix.workload()[1] <= once.workload()[1]


@pytest.mark.parametrize("seed", range(12))
def test_fixpoint_is_exact_for_trees_with_distinct_labels(seed):
    """For a tree query whose labels are pairwise distinct, the fixpoint's
    C(u) is exactly the set of images of u over all embeddings: on a tree,
    arc consistency leaves only values that extend to a homomorphism, and
    distinct labels make every homomorphism injective."""
    rng = np.random.default_rng(700 + seed)
    n, L = 150, 6
    edges, labels = random_graph(rng, n, 0.06, L)
    k = int(rng.integers(2, 6))
    ql = rng.permutation(L)[:k].astype(np.int32)
    qe = np.array([[int(rng.integers(0, v)), v] for v in range(1, k)], np.int32)
    g = oracle.Graph(n, edges, labels)
    fix = oracle.Cst(g, ql, qe, refine="fixpoint")
    r = oracle.match(g, ql, qe, max_emb=1 << 20)
    assert r["complete"] and r["count"] < 1 << 20
    for u in range(k):
        proj = set(r["emb"][:, u].tolist()) if r["count"] else set()
        assert set(fix.cand(u).tolist()) == proj, u


def test_once_with_non_tree_test_hand_case():
    """Triangle query A-B-C rooted at A (non-tree edge B-C).  G holds the
    triangle a1 b1 c1 and a path b2 - a2 - c2 whose b2 and c2 are not
    adjacent (each has one more neighbour, so the degree filter keeps them).
    One pass keeps a2, b2 and c2; the pass with the non-tree test removes c2
    and b2 (no neighbour among the other's candidates), and then a2, whose
    list into B is empty."""
    e = np.array([(0, 1), (0, 2), (1, 2), (3, 4), (3, 5), (4, 6), (5, 7)], np.int32)
    lab = np.array([0, 1, 2, 0, 1, 2, 3, 3], np.int32)
    g = oracle.Graph(8, e, lab)
    ql, qe = np.array([0, 1, 2], np.int32), np.array([(0, 1), (0, 2), (1, 2)], np.int32)
    once = oracle.Cst(g, ql, qe)
    nt = oracle.Cst(g, ql, qe, refine="once_nt")
    assert once.root == nt.root == 0
    assert [once.cand(u).tolist() for u in range(3)] == [[0, 3], [1, 4], [2, 5]]
    assert [nt.cand(u).tolist() for u in range(3)] == [[0], [1], [2]]
    assert oracle.count(g, ql, qe) == 1


@pytest.mark.parametrize("seed", range(25))
def test_once_with_non_tree_test_lies_between(seed):
    """The single pass with the non-tree test keeps every embedding's images
    and lies between the fixpoint and the paper's single pass, vertex by
    vertex (same root and t_q)."""
    n, edges, labels, ql, qe = _cst_case(seed)
    g = oracle.Graph(n, edges, labels)
    once = oracle.Cst(g, ql, qe)
    nt = oracle.Cst(g, ql, qe, refine="once_nt")
    fix = oracle.Cst(g, ql, qe, refine="fixpoint")
    k = len(ql)
    assert nt.root == once.root and nt.parent.tolist() == once.parent.tolist()
    for u in range(k):
        a, b, c = set(fix.cand(u).tolist()), set(nt.cand(u).tolist()), set(once.cand(u).tolist())
        assert a <= b <= c, u
    r = oracle.match(g, ql, qe, max_emb=1 << 18)
    for row in r["emb"].tolist():
        for u in range(k):
            assert row[u] in set(nt.cand(u).tolist())
    assert r["count"] <= nt.workload()[1] <= once.workload()[1]
