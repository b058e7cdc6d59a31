"""ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain, slow CPU implementations of what the subgraph-matching path computes,
used to check the CUDA library.  Only the test suite, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import this package; the library
(``paper_2102_10768_gb300``) never does, and the two share no code.

* ``oracle.c``   -- the data graph and a backtracking enumerator of every
                    embedding (Definition 1 and the problem statement of
                    Sec. II-A), with optional allowed sets per query vertex.
* ``cst_ref.c``  -- the candidate search tree of Algorithm 1 (Sec. IV-A), the
                    query preparation it needs, and the workload estimate of
                    Sec. IV-C.
* ``brute_force`` (here) -- every injective map, tried one by one; tiny inputs
                    only.  It pins the backtracker.

Parity status: the enumerator is pinned by brute force, closed forms and the
automorphism invariant; the CST restatement by the soundness theorem of
Sec. IV-A and by a hand-built fixture for the workload example of Sec. IV-C.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "cst_ref.c")]
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into _build/liboracle.so."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _SO] + _SRCS)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        lib.oracle_graph_new.argtypes = [i64, i64, vp, vp]
        lib.oracle_graph_new.restype = vp
        lib.oracle_graph_free.argtypes = [vp]
        lib.oracle_graph_nadj.argtypes = [vp]
        lib.oracle_graph_nadj.restype = i64
        lib.oracle_graph_csr.argtypes = [vp, vp, vp]
        lib.oracle_match.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                     i64, vp, vp, vp, vp, i64, ctypes.c_int, u64]
        lib.oracle_check_embeddings.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, i64, vp]
        lib.oracle_check_embeddings.restype = i64
        lib.oracle_cst_build.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int]
        lib.oracle_cst_build.restype = vp
        lib.oracle_cst_free.argtypes = [vp]
        lib.oracle_cst_root.argtypes = [vp]
        lib.oracle_cst_tree_shape.argtypes = [vp, vp, vp, vp]
        lib.oracle_cst_c0_count.argtypes = [vp, ctypes.c_int]
        lib.oracle_cst_c0_count.restype = i64
        lib.oracle_cst_cand_count.argtypes = [vp, ctypes.c_int]
        lib.oracle_cst_cand_count.restype = i64
        lib.oracle_cst_cand.argtypes = [vp, ctypes.c_int, vp]
        lib.oracle_cst_tree_total.argtypes = [vp, ctypes.c_int]
        lib.oracle_cst_tree_total.restype = i64
        lib.oracle_cst_tree.argtypes = [vp, ctypes.c_int, vp, vp]
        lib.oracle_cst_nt_count.argtypes = [vp]
        lib.oracle_cst_nt_edge.argtypes = [vp, ctypes.c_int, vp, vp]
        lib.oracle_cst_nt_total.argtypes = [vp, ctypes.c_int]
        lib.oracle_cst_nt_total.restype = i64
        lib.oracle_cst_nt.argtypes = [vp, ctypes.c_int, vp, vp]
        lib.oracle_cst_workload.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp]
        lib.oracle_cst_partition.argtypes = [vp, u64, ctypes.c_double, ctypes.c_double, u64, i64,
                                             vp, vp, vp, vp, vp, vp]
        lib.oracle_cst_partition.restype = i64
        lib.oracle_cst_chunk_w.argtypes = [vp, ctypes.c_int, vp, vp, i64]
        lib.oracle_cst_chunk_w.restype = u64
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class Graph:
    """Simple undirected labelled data graph (loops and repeats dropped)."""

    def __init__(self, n: int, edges, labels):
        self.n = int(n)
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
        assert lab.shape[0] == self.n
        self.labels = lab
        self._h = _L().oracle_graph_new(self.n, e.shape[0], _p(e), _p(lab))
        if not self._h:
            raise ValueError("oracle: bad edge list")

    def csr(self):
        nadj = _L().oracle_graph_nadj(self._h)
        off = np.empty(self.n + 1, dtype=np.int64)
        adj = np.empty(max(nadj, 1), dtype=np.int32)
        _L().oracle_graph_csr(self._h, _p(off), _p(adj))
        return off, adj[:nadj]

    def close(self):
        if getattr(self, "_h", None):
            _L().oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


def _qarrays(qlabels, qedges):
    ql = np.ascontiguousarray(np.asarray(qlabels, dtype=np.int32))
    qe = np.ascontiguousarray(np.asarray(qedges, dtype=np.int32).reshape(-1, 2))
    return ql, qe


def match(g: Graph, qlabels, qedges, order=None, par=None, allow=None, max_emb: int = 0,
          budget: int = 0, threads: int = 0, want_depth: bool = False, want_balg: bool = False,
          limit: int = 0):
    """Enumerate embeddings of q in G by plain backtracking (Definition 1).

    allow: optional {query vertex: iterable of allowed data vertices}.
    limit: stop after `limit` embeddings (count = min(total, limit)).
    Returns a dict: count, complete (False if the per-thread node budget was
    hit), emb (sorted int32[rows][k] indexed by query vertex, at most
    max_emb rows), depth (partial results per number of mapped positions),
    balg / balg_max: floor and ceiling of the bytes a search over the CST
    requests (see oracle_match in oracle.c).
    """
    ql, qe = _qarrays(qlabels, qedges)
    k = ql.shape[0]
    o = None if order is None else np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    pp = None if par is None else np.ascontiguousarray(np.asarray(par, dtype=np.int32))
    aoff = av = aon = None
    if allow:
        aon = np.zeros(k, dtype=np.uint8)
        parts = []
        aoff = np.zeros(k + 1, dtype=np.int64)
        for u in range(k):
            s = np.unique(np.asarray(list(allow[u]) if u in allow else [], dtype=np.int32))
            if u in allow:
                aon[u] = 1
            parts.append(s)
            aoff[u + 1] = aoff[u] + s.shape[0]
        av = np.ascontiguousarray(np.concatenate(parts).astype(np.int32)) if aoff[-1] else np.zeros(1, np.int32)
    emb = np.zeros((max(max_emb, 1), k), dtype=np.int32)
    cnt = np.zeros(1, dtype=np.uint64)
    depth = np.zeros(k, dtype=np.uint64)
    balg = np.zeros(2, dtype=np.float64)
    rc = _L().oracle_match(g._h, k, _p(ql), qe.shape[0], _p(qe), _p(o), _p(pp), _p(aoff), _p(av), _p(aon),
                           max_emb, _p(emb), _p(cnt), _p(depth), _p(balg) if want_balg else None,
                           budget, threads, limit)
    if rc < 0:
        raise ValueError(f"oracle_match: invalid input ({rc})")
    count = int(cnt[0])
    rows = emb[:min(count, max_emb)] if max_emb > 0 else emb[:0]
    if rows.shape[0]:
        rows = rows[np.lexsort(rows.T[::-1])]
    return {"count": count, "complete": rc == 0, "emb": rows,
            "depth": depth.astype(np.int64) if want_depth else None,
            "balg": float(balg[0]) if want_balg else None,
            "balg_max": float(balg[1]) if want_balg else None}


def invalid_rows(g: Graph, qlabels, qedges, emb) -> int:
    """How many rows of emb[rows][k] (by query vertex) are not embeddings
    of q in G by Definition 1."""
    ql, qe = _qarrays(qlabels, qedges)
    e = np.ascontiguousarray(np.asarray(emb, dtype=np.int32).reshape(-1, ql.shape[0]))
    return int(_L().oracle_check_embeddings(g._h, ql.shape[0], _p(ql), qe.shape[0], _p(qe), e.shape[0], _p(e)))


def count(g: Graph, qlabels, qedges, **kw) -> int:
    r = match(g, qlabels, qedges, **kw)
    assert r["complete"]
    return r["count"]


class Cst:
    """Candidate search tree of Algorithm 1, restated on the CPU."""

    ORDERS = {"path": 0, "greedy": 1, "bfs": 2, "mincand": 3}
    FILTERS = {"ldf": 0, "nlf": 1}
    REFINES = {"once": 0, "fixpoint": 1, "once_nt": 2}

    def __init__(self, g: Graph, qlabels, qedges, order: str = "path", filter: str = "ldf", refine: str = "once"):
        """order: "path" (the paper's path-based order), "greedy" (edges
        to already placed vertices first), "bfs" (the BFS order of t_q) or
        "mincand" (the placeable vertex with the fewest candidates); filter: "ldf" (label and degree)
        or "nlf" (also neighbour label frequencies); refine: "once" (the
        paper's single bottom-up pass), "fixpoint" (repeated, with the
        non-tree neighbour test) or "once_nt" (one pass with that test); see
        oracle/cst_ref.c."""
        ql, qe = _qarrays(qlabels, qedges)
        self.k = ql.shape[0]
        self._h = _L().oracle_cst_build(g._h, self.k, _p(ql), qe.shape[0], _p(qe), self.ORDERS[order],
                                        self.FILTERS[filter], self.REFINES[refine])
        if not self._h:
            raise ValueError("oracle_cst_build: invalid or disconnected query")
        k = self.k
        self.root = _L().oracle_cst_root(self._h)
        par = np.empty(k, np.int32); bfs = np.empty(k, np.int32); order = np.empty(k, np.int32)
        _L().oracle_cst_tree_shape(self._h, _p(par), _p(bfs), _p(order))
        self.parent, self.bfs, self.order = par, bfs, order
        self.c0_count = np.array([_L().oracle_cst_c0_count(self._h, u) for u in range(k)], np.int64)

    def cand(self, u: int) -> np.ndarray:
        n = _L().oracle_cst_cand_count(self._h, u)
        out = np.empty(max(n, 1), np.int32)
        _L().oracle_cst_cand(self._h, u, _p(out))
        return out[:n]

    def tree(self, u: int):
        """Lists N^{p(u)}_u(v_p) for v_p in C(p(u)): (offsets, global ids)."""
        rows = self.cand(int(self.parent[u])).shape[0]
        tot = _L().oracle_cst_tree_total(self._h, u)
        off = np.empty(rows + 1, np.int64)
        vals = np.empty(max(tot, 1), np.int32)
        _L().oracle_cst_tree(self._h, u, _p(off), _p(vals))
        return off, vals[:tot]

    def nontree(self):
        """[(from_u, to_u, offsets, global ids)] for each non-tree edge,
        from the earlier to the later endpoint in the matching order."""
        out = []
        for e in range(_L().oracle_cst_nt_count(self._h)):
            a = np.zeros(1, np.int32); b = np.zeros(1, np.int32)
            _L().oracle_cst_nt_edge(self._h, e, _p(a), _p(b))
            rows = self.cand(int(a[0])).shape[0]
            tot = _L().oracle_cst_nt_total(self._h, e)
            off = np.empty(rows + 1, np.int64)
            vals = np.empty(max(tot, 1), np.int32)
            _L().oracle_cst_nt(self._h, e, _p(off), _p(vals))
            out.append((int(a[0]), int(b[0]), off, vals[:tot]))
        return out

    def workload(self, dump_u: int = -1):
        """(W as float64, W as saturating uint64, c_u(v) float64, c_u(v) uint64)."""
        wf = np.zeros(1, np.float64); wi = np.zeros(1, np.uint64)
        n = self.cand(dump_u).shape[0] if dump_u >= 0 else 0
        cf = np.zeros(max(n, 1), np.float64); ci = np.zeros(max(n, 1), np.uint64)
        _L().oracle_cst_workload(self._h, _p(wf), _p(wi), dump_u, _p(cf), _p(ci))
        return float(wf[0]), int(wi[0]), cf[:n], ci[:n]

    def partition(self, delta_w: int, c_root: float = 0.0, c_deep: float = 0.0, seed: int = 0,
                  max_chunks: int = 1 << 16):
        """Algorithm 2 (readings in cst_ref.c).  Returns a list of chunks
        (j, prefix global ids tuple, a, b, W', id), level by level."""
        k = self.k
        j = np.empty(max_chunks, np.int32); pre = np.empty((max_chunks, k), np.int32)
        a = np.empty(max_chunks, np.int64); b = np.empty(max_chunks, np.int64)
        w = np.empty(max_chunks, np.uint64); ids = np.empty(max_chunks, np.uint64)
        n = _L().oracle_cst_partition(self._h, int(delta_w), float(c_root), float(c_deep), int(seed),
                                      max_chunks, _p(j), _p(pre), _p(a), _p(b), _p(w), _p(ids))
        if n < 0:
            raise OverflowError("oracle partition: more than max_chunks chunks")
        return [(int(j[i]), tuple(int(x) for x in pre[i, :j[i]]), int(a[i]), int(b[i]), int(w[i]), int(ids[i]))
                for i in range(n)]

    def chunk_list(self, j: int, prefix):
        """L_j of a chunk: C(root) for j = 0, else the tree list of the
        prefix candidate at position j's parent position (global ids)."""
        u = int(self.order[j])
        if j == 0:
            return self.cand(u)
        p = int(self.parent[u])
        pos = {int(x): i for i, x in enumerate(self.order)}
        cp = self.cand(p)
        row = int(np.searchsorted(cp, prefix[pos[p]]))
        off, vals = self.tree(u)
        return vals[off[row]:off[row + 1]]

    def chunk_w(self, j: int, prefix, run) -> int:
        pre = np.ascontiguousarray(np.asarray(list(prefix) + [0], dtype=np.int32))
        r = np.ascontiguousarray(np.asarray(run, dtype=np.int32))
        return int(_L().oracle_cst_chunk_w(self._h, j, _p(pre), _p(r) if r.size else None, r.shape[0]))

    def chunk_allow(self, j: int, prefix, a: int, b: int):
        """Allowed sets that confine the enumerator to one chunk."""
        allow = {int(self.order[i]): [int(prefix[i])] for i in range(j)}
        allow[int(self.order[j])] = self.chunk_list(j, prefix)[a:b].tolist()
        return allow

    def close(self):
        if getattr(self, "_h", None):
            _L().oracle_cst_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


def brute_force(n: int, edges, labels, qlabels, qedges):
    """Every injective map V(q) -> V(G), tested one by one against
    Definition 1.  Returns the sorted list of embeddings (tuples indexed by
    query vertex).  Tiny inputs only: n!/(n-k)! maps."""
    E = set()
    for a, b in np.asarray(edges).reshape(-1, 2).tolist():
        if a != b:
            E.add((a, b)); E.add((b, a))
    lab = list(np.asarray(labels).tolist())
    ql = list(np.asarray(qlabels).tolist())
    qe = np.asarray(qedges).reshape(-1, 2).tolist()
    out = []
    for M in itertools.permutations(range(n), len(ql)):
        if all(lab[M[u]] == ql[u] for u in range(len(ql))) and all((M[a], M[b]) in E for a, b in qe):
            out.append(M)
    return sorted(out)
