"""Seeded synthetic graphs and queries for the subgraph-matching workloads.

The generators live in ``gen.c`` (built into ``_build/libsynth.so`` by
:func:`build`); this module only marshals arrays.  Nothing here filters,
searches or counts: both the CUDA library and the CPU oracle take their
inputs from here and from nowhere else.

Workload recipes (the data graphs stand in for the paper's LDBC-SNB datasets,
Tab. III, and the random-walk queries for its query set, Fig. 5, neither of
which is available):

* ``er_workload``      -- Erdos-Renyi G(n=10,000, m=40,000), 8 uniform labels,
                          8 connected 4-vertex induced random-walk queries.
* ``powerlaw_workload``-- Chung-Lu, exponent 2.1, 1M vertices, 16M edges,
                          16 Zipf(1.0) labels; dense and sparse random-walk
                          queries of 8 and 16 vertices.
* ``rmat_graph``       -- R-MAT(a=.57, b=c=.19), any scale.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None

KIND = {"induced": 0, "dense": 1, "sparse": 2}


def build(force: bool = False) -> str:
    """Compile gen.c into _build/libsynth.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _SO, src, "-lm"])
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, u64, i32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p
        lib.synth_er_edges.argtypes = [i64, i64, u64, vp]
        lib.synth_chung_lu_edges.argtypes = [i64, i64, ctypes.c_double, u64, vp]
        lib.synth_rmat_edges.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, u64, vp]
        lib.synth_labels_uniform.argtypes = [i64, i32, u64, vp]
        lib.synth_labels_zipf.argtypes = [i64, i32, ctypes.c_double, u64, vp]
        lib.synth_walk_graph_new.argtypes = [i64, i64, vp]
        lib.synth_walk_graph_new.restype = vp
        lib.synth_walk_graph_free.argtypes = [vp]
        lib.synth_walk_query.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, u64, u64, ctypes.c_int,
                                         vp, vp, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc < 0:
        raise RuntimeError(f"synth: {what} failed with code {rc}")


def er_edges(n: int, m: int, seed: int) -> np.ndarray:
    out = np.empty((m, 2), dtype=np.int32)
    _check(_L().synth_er_edges(n, m, seed, _ptr(out)), "er_edges")
    return out


def chung_lu_edges(n: int, m: int, gamma: float, seed: int) -> np.ndarray:
    out = np.empty((m, 2), dtype=np.int32)
    _check(_L().synth_chung_lu_edges(n, m, gamma, seed, _ptr(out)), "chung_lu_edges")
    return out


def rmat_edges(scale: int, m: int, seed: int, a=0.57, b=0.19, c=0.19) -> np.ndarray:
    out = np.empty((m, 2), dtype=np.int32)
    _check(_L().synth_rmat_edges(scale, m, a, b, c, seed, _ptr(out)), "rmat_edges")
    return out


def labels_uniform(n: int, L: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _check(_L().synth_labels_uniform(n, L, seed, _ptr(out)), "labels_uniform")
    return out


def labels_zipf(n: int, L: int, seed: int, s: float = 1.0) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _check(_L().synth_labels_zipf(n, L, s, seed, _ptr(out)), "labels_zipf")
    return out


@dataclass
class Query:
    """A connected labelled query graph; ``verts`` is the walk it came from
    (query vertex i was drawn from data vertex verts[i])."""
    labels: np.ndarray            # int32[k]
    edges: np.ndarray             # int32[m][2], each unordered pair once
    verts: np.ndarray = field(default=None)
    kind: str = "induced"

    @property
    def k(self) -> int:
        return int(self.labels.shape[0])

    @property
    def avg_degree(self) -> float:
        return 2.0 * self.edges.shape[0] / max(self.k, 1)


class WalkGraph:
    """Host adjacency used only to draw random walks."""

    def __init__(self, n: int, edges: np.ndarray):
        edges = np.ascontiguousarray(edges, dtype=np.int32)
        self.n = n
        self._h = _L().synth_walk_graph_new(n, edges.shape[0], _ptr(edges))
        if not self._h:
            raise MemoryError("synth_walk_graph_new")

    def close(self):
        if self._h:
            _L().synth_walk_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def query(self, labels: np.ndarray, k: int, kind: str, seed: int, stream: int,
              max_attempts: int = 10000) -> Query:
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        verts = np.empty(k, dtype=np.int32)
        ql = np.empty(k, dtype=np.int32)
        qe = np.empty((max(k * (k - 1) // 2, 1), 2), dtype=np.int32)
        rc = _L().synth_walk_query(self._h, _ptr(labels), k, KIND[kind], seed, stream,
                                   max_attempts, _ptr(verts), _ptr(ql), _ptr(qe))
        _check(rc, f"walk_query(k={k}, kind={kind})")
        return Query(labels=ql, edges=qe[:rc].copy(), verts=verts, kind=kind)


def walk_queries(n: int, edges: np.ndarray, labels: np.ndarray, k: int, count: int, kind: str,
                 seed: int, stream0: int = 0) -> list[Query]:
    wg = WalkGraph(n, edges)
    try:
        return [wg.query(labels, k, kind, seed, stream0 + j) for j in range(count)]
    finally:
        wg.close()


def kinds_for(k: int) -> tuple:
    """The two query kinds drawn at size k: dense and sparse, except that a
    4-vertex query cannot have average degree > 3, so 4-vertex queries are
    induced and sparse."""
    return ("induced", "sparse") if k == 4 else ("dense", "sparse")


def mixed_queries(wg: "WalkGraph", labels: np.ndarray, sizes, per_size: int, seed: int) -> list:
    """per_size random-walk queries of each size in `sizes`, the two kinds of
    kinds_for(k) alternating, walk j of size k drawn from stream
    100,000 * k + j: a list of (labels, edges)."""
    qs = []
    for k in sizes:
        kinds = kinds_for(k)
        for j in range(per_size):
            q = wg.query(labels, k, kinds[j % 2], seed, 100_000 * k + j)
            qs.append((q.labels, q.edges))
    return qs


# ----------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    n: int
    edges: np.ndarray             # int32[m][2]
    labels: np.ndarray            # int32[n]
    queries: list
    num_labels: int


def er_workload(seed: int = 1000) -> Workload:
    """10,000-vertex Erdos-Renyi graph with 40,000 edges (average degree 8),
    8 uniform labels, and 8 connected 4-vertex induced random-walk queries."""
    n, m, L = 10_000, 40_000, 8
    e = er_edges(n, m, seed)
    lab = labels_uniform(n, L, seed)
    qs = walk_queries(n, e, lab, 4, 8, "induced", seed)
    return Workload("er-10k-40k-L8-q4x8", n, e, lab, qs, L)


def powerlaw_graph(seed: int = 2000, n: int = 1_000_000, m: int = 16_000_000, gamma: float = 2.1,
                   L: int = 16):
    e = chung_lu_edges(n, m, gamma, seed)
    lab = labels_zipf(n, L, seed)
    return n, e, lab


def rmat_graph(scale: int, edge_factor: int, L: int, seed: int):
    n = 1 << scale
    e = rmat_edges(scale, edge_factor * n, seed)
    lab = labels_zipf(n, L, seed)
    return n, e, lab
