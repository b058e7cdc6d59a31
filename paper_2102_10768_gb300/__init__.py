"""GB300 candidate-search-tree subgraph matching (after arXiv 2102.10768).

A thin binding of the C ABI in ``include/fast.h`` (``_build/libfast.so``):
argument marshalling only -- every step of the computation runs in the
library's CUDA kernels.  PyTorch, when present, only supplies the current
CUDA stream and device buffers.  The library must be built (``build()``);
importing this module without it raises.

Low-level functions keep the C names (``fast_load_graph`` ...); the classes
``Graph``, ``Cst`` and ``Chunks`` own the corresponding handles.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FAST_OK = 0
FAST_ERR_INVALID = 1
FAST_ERR_OOM = 2
FAST_ERR_TIMEOUT = 3
FAST_ERR_OVERFLOW = 4
FAST_ERR_CUDA = 5
FAST_ERR_LIMIT = 6
FAST_PTR_DEVICE = 1
FAST_MAX_QUERY = 32

_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "TIMEOUT", 4: "OVERFLOW", 5: "CUDA", 6: "LIMIT"}


class FastError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"FAST_ERR_{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    __slots__ = ()              # a misspelled field raises instead of being ignored
    _fields_ = [("delta_w", ctypes.c_uint64), ("sample_root", ctypes.c_double),
                ("sample_deep", ctypes.c_double), ("sample_seed", ctypes.c_uint64),
                ("max_chunks", ctypes.c_int64), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("time_budget_s", ctypes.c_double),
                ("limit", ctypes.c_uint64), ("queue_cells", ctypes.c_int64), ("order_rule", ctypes.c_int32),
                ("filter_rule", ctypes.c_int32), ("build_rule", ctypes.c_int32), ("refine_rule", ctypes.c_int32),
                ("matcher_rule", ctypes.c_int32), ("validators", ctypes.c_int32)]


class QueryDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32),
                ("labels", ctypes.POINTER(ctypes.c_int32)), ("edges", ctypes.POINTER(ctypes.c_int32))]


_lib = None
_vp = ctypes.c_void_p
_i64, _i32, _u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64

_SIGS = {
    "fast_config_default": (None, [_vp]),
    "fast_last_error": (ctypes.c_char_p, []),
    "fast_load_graph": (ctypes.c_int, [_i64, _i64, _vp, _vp, ctypes.c_int, _vp, _vp]),
    "fast_graph_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fast_graph_copy_csr": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fast_free_graph": (None, [_vp]),
    "fast_build_cst": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fast_build_cst_batch": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "fast_partition_batch": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "fast_inject_alloc_failure": (ctypes.c_int64, [_i64]),
    "fast_cst_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fast_cst_candidates": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "fast_cst_tree_size": (ctypes.c_int, [_vp, _i32, _vp]),
    "fast_cst_tree_lists": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fast_cst_nontree_count": (ctypes.c_int, [_vp, _vp]),
    "fast_cst_nontree_edge": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fast_cst_nontree_lists": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fast_cst_workload": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "fast_free_cst": (None, [_vp]),
    "fast_partition": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fast_chunks_info": (ctypes.c_int, [_vp, _vp, _vp]),
    "fast_chunks_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fast_free_chunks": (None, [_vp]),
    "fast_match": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _vp, _vp]),
    "fast_match_ex": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp, _vp]),
    "fast_match_stats": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fast_batch_create": (ctypes.c_int, [_vp, _vp, _i32, _i32, _vp]),
    "fast_batch_run": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "fast_batch_timing": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fast_batch_config": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "fast_batch_autotune": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fast_free_batch": (None, [_vp]),
    "fast_match_batch": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "fast_server_create": (ctypes.c_int, [_vp, _vp, _u64, _i32, _vp]),
    "fast_server_submit": (ctypes.c_int, [_vp, _vp, _vp]),
    "fast_server_poll": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32]),
    "fast_server_groups": (ctypes.c_int, [_vp, _vp, _vp]),
    "fast_batch_bytes": (ctypes.c_int, [_vp, _vp, _vp]),
    "fast_chunks_select": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "fast_last_match_floor_bytes": (ctypes.c_uint64, []),
    "fast_server_stats": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fast_server_destroy": (None, [_vp]),
    "fast_now_ns": (ctypes.c_uint64, []),
    "fast_match_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp]),
    "fast_match_noalloc_scratch_bytes": (ctypes.c_uint64, []),
    "fast_last_match_ms": (ctypes.c_double, []),
    "fast_last_match_bytes": (ctypes.c_uint64, []),
    "fast_kernel_launches": (ctypes.c_uint64, []),
    "fast_last_build_round_trips": (ctypes.c_uint64, []),
}


def build(force: bool = False) -> str:
    """Compile the CUDA library (sm_103a) in-tree."""
    return _build.build(force=force)


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libfast.so; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build the CUDA library first "
                               "(paper_2102_10768_gb300.build())")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int):
    if rc != FAST_OK:
        raise FastError(rc, lib().fast_last_error().decode())


def _p(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a


def default_stream():
    """cudaStream_t of torch's current stream (None = legacy default)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def inject_alloc_failure(after: int) -> int:
    """fast_inject_alloc_failure: the next `after` device allocations succeed,
    the one after them fails with FAST_ERR_OOM (once); after < 0: off.
    Returns the replaced countdown (-1: the failure has happened, or was off)."""
    return lib().fast_inject_alloc_failure(after)


def default_config(**kw) -> Config:
    """fast_config_default, then the given fields (unknown names raise)."""
    c = Config()
    lib().fast_config_default(ctypes.byref(c))
    fields = {f[0] for f in Config._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError(f"fast_config has no field {k!r}")
        setattr(c, k, v)
    return c


# ------------------------------------------------------------------ handles

class Graph:
    """Device-resident data graph (fast_load_graph)."""

    def __init__(self, n: int, edges, labels, stream=None, device: bool = False):
        self.n = int(n)
        self._keep = None
        if device:
            e, lab = edges, labels
            m = int(edges.shape[0])
        else:
            e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
            lab = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
            m = e.shape[0]
        h = _vp()
        st = stream if stream is not None else default_stream()
        _check(lib().fast_load_graph(self.n, m, _p(e), _p(lab), FAST_PTR_DEVICE if device else 0, st,
                                     ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nadj, ml = _i64(), _i64(), _i64()
        nl = _i32()
        _check(lib().fast_graph_info(self._h, ctypes.byref(n), ctypes.byref(nadj), ctypes.byref(nl), ctypes.byref(ml)))
        return {"n": n.value, "nadj": nadj.value, "num_labels": nl.value, "max_degree": ml.value}

    def csr(self, stream=None):
        inf = self.info()
        off = np.empty(inf["n"] + 1, np.int64)
        col = np.empty(max(inf["nadj"], 1), np.int32)
        _check(lib().fast_graph_copy_csr(self._h, _p(off), _p(col), stream if stream is not None else default_stream()))
        return off, col[:inf["nadj"]]

    def close(self):
        if getattr(self, "_h", None):
            lib().fast_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cst:
    """Candidate search tree of one query (fast_build_cst)."""

    def __init__(self, graph: Graph, qlabels, qedges, cfg: Config | None = None, stream=None):
        ql = np.ascontiguousarray(np.asarray(qlabels, dtype=np.int32))
        qe = np.ascontiguousarray(np.asarray(qedges, dtype=np.int32).reshape(-1, 2))
        self.graph = graph
        self.k = int(ql.shape[0])
        self._ql, self._qe = ql, qe
        q = QueryDesc(self.k, qe.shape[0], ql.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      qe.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        h = _vp()
        self.stream = stream if stream is not None else default_stream()
        _check(lib().fast_build_cst(graph.handle, ctypes.byref(q), ctypes.byref(cfg) if cfg else None,
                                    self.stream, ctypes.byref(h)))
        self._h = h
        self._load_info()

    @classmethod
    def _adopt(cls, graph: Graph, ql, qe, h, stream):
        """Wraps a CST handle that the library built (fast_build_cst_batch)."""
        self = cls.__new__(cls)
        self.graph = graph
        self.k = int(ql.shape[0])
        self._ql, self._qe = ql, qe
        self.stream = stream
        self._h = h
        self._load_info()
        return self

    def _load_info(self):
        h = self._h
        k = self.k
        kk, root = _i32(), _i32()
        order = np.empty(k, np.int32); parent = np.empty(k, np.int32); cand = np.empty(k, np.int64)
        wu, wf = _u64(), ctypes.c_double()
        _check(lib().fast_cst_info(h, ctypes.byref(kk), ctypes.byref(root), _p(order), _p(parent), _p(cand),
                                   ctypes.byref(wu), ctypes.byref(wf)))
        self.root, self.order, self.parent, self.ncand = root.value, order, parent, cand
        self.W, self.Wf = wu.value, wf.value

    @property
    def handle(self):
        return self._h

    def candidates(self, u: int) -> np.ndarray:
        out = np.empty(max(int(self.ncand[u]), 1), np.int32)
        _check(lib().fast_cst_candidates(self._h, u, _p(out), self.stream))
        return out[:int(self.ncand[u])]

    def tree_lists(self, u: int):
        """(offsets over C(parent(u)), candidate-local indices into C(u))."""
        ent = _i64()
        _check(lib().fast_cst_tree_size(self._h, u, ctypes.byref(ent)))
        rows = int(self.ncand[int(self.parent[u])])
        off = np.empty(rows + 1, np.int64)
        idx = np.empty(max(ent.value, 1), np.uint32)
        _check(lib().fast_cst_tree_lists(self._h, u, _p(off), _p(idx), self.stream))
        return off, idx[:ent.value]

    def nontree(self):
        """[(from_u, to_u, offsets, candidate-local indices into C(to_u))]."""
        cnt = _i32()
        _check(lib().fast_cst_nontree_count(self._h, ctypes.byref(cnt)))
        out = []
        for e in range(cnt.value):
            a, b, ent = _i32(), _i32(), _i64()
            _check(lib().fast_cst_nontree_edge(self._h, e, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ent)))
            rows = int(self.ncand[a.value])
            off = np.empty(rows + 1, np.int64)
            idx = np.empty(max(ent.value, 1), np.uint32)
            _check(lib().fast_cst_nontree_lists(self._h, e, _p(off), _p(idx), self.stream))
            out.append((a.value, b.value, off, idx[:ent.value]))
        return out

    def workload(self, u: int) -> np.ndarray:
        out = np.empty(max(int(self.ncand[u]), 1), np.uint64)
        _check(lib().fast_cst_workload(self._h, u, _p(out), self.stream))
        return out[:int(self.ncand[u])]

    def close(self):
        if getattr(self, "_h", None):
            lib().fast_free_cst(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chunks:
    """Partition of a CST (fast_partition)."""

    def __init__(self, cst: Cst, cfg: Config | None = None, stream=None):
        self.cst = cst
        h = _vp()
        self.stream = stream if stream is not None else cst.stream
        _check(lib().fast_partition(cst.handle, ctypes.byref(cfg) if cfg else None, self.stream, ctypes.byref(h)))
        self._h = h
        self._load_info()

    @classmethod
    def _adopt(cls, cst: Cst, h, stream):
        """Wraps a chunk list that the library built (fast_partition_batch)."""
        self = cls.__new__(cls)
        self.cst = cst
        self.stream = stream
        self._h = h
        self._load_info()
        return self

    def _load_info(self):
        n, ws = _i64(), _u64()
        _check(lib().fast_chunks_info(self._h, ctypes.byref(n), ctypes.byref(ws)))
        self.n, self.w_sum = n.value, ws.value

    @property
    def handle(self):
        return self._h

    def copy(self):
        """List of (j, prefix tuple of candidate-local indices, a, b, W', id)."""
        n, k = self.n, self.cst.k
        j = np.empty(max(n, 1), np.int32); pre = np.empty((max(n, 1), k), np.int32)
        a = np.empty(max(n, 1), np.int64); b = np.empty(max(n, 1), np.int64)
        w = np.empty(max(n, 1), np.uint64); ids = np.empty(max(n, 1), np.uint64)
        _check(lib().fast_chunks_copy(self._h, _p(j), _p(pre), _p(a), _p(b), _p(w), _p(ids), self.stream))
        return [(int(j[i]), tuple(int(x) for x in pre[i, :j[i]]), int(a[i]), int(b[i]), int(w[i]), int(ids[i]))
                for i in range(n)]

    def weights(self) -> np.ndarray:
        """W' of every chunk (uint64)."""
        n = self.n
        w = np.empty(max(n, 1), np.uint64)
        _check(lib().fast_chunks_copy(self._h, None, None, None, None, _p(w), None, self.stream))
        return w[:n]

    def select(self, idx) -> "Chunks":
        """fast_chunks_select: the chunks idx (host indices, in order) as a new
        list over the same CST -- one rank's share of a sharded query."""
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
        h = _vp()
        _check(lib().fast_chunks_select(self._h, _p(ix) if ix.size else None, ix.size, self.stream, ctypes.byref(h)))
        return Chunks._adopt(self.cst, h, self.stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().fast_free_chunks(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match(cst: Cst, chunks: Chunks | None = None, k: int = 0, emb_out=None, cfg: Config | None = None,
          chunk_counts=None, stream=None, check: bool = True):
    """fast_match_ex.  emb_out: device tensor / host array with >= k rows of
    cst.k uint32 (allocated on the host here when None and k > 0).
    chunk_counts: optional device buffer of one uint64 per chunk.
    Returns dict(count, written, status, emb)."""
    if k > 0 and emb_out is None:
        emb_out = np.zeros((k, cst.k), np.uint32)
    cnt, wr = _u64(), _u64()
    rc = lib().fast_match_ex(cst.handle, chunks.handle if chunks else None, ctypes.byref(cfg) if cfg else None,
                             k, _p(emb_out), ctypes.byref(cnt), ctypes.byref(wr), _p(chunk_counts),
                             stream if stream is not None else cst.stream)
    if check and rc not in (FAST_OK,):
        _check(rc)
    return {"count": cnt.value, "written": wr.value, "status": rc, "emb": emb_out}


def _query_descs(queries):
    """ctypes array of QueryDesc for [(labels, edges)], plus the arrays it points to."""
    keep = []
    arr = (QueryDesc * max(len(queries), 1))()
    for i, (ql, qe) in enumerate(queries):
        ql = np.ascontiguousarray(np.asarray(ql, dtype=np.int32))
        qe = np.ascontiguousarray(np.asarray(qe, dtype=np.int32).reshape(-1, 2))
        keep += [ql, qe]
        arr[i] = QueryDesc(ql.shape[0], qe.shape[0], ql.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           qe.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return arr, keep


def build_csts(graph: Graph, queries, cfg: Config | None = None, stream=None):
    """CSTs of many queries built together (fast_build_cst_batch): a list with
    a Cst per query (None where the query is invalid) and the status array."""
    arr, keep = _query_descs(queries)
    nq = len(queries)
    outs = (_vp * max(nq, 1))()
    status = np.zeros(max(nq, 1), np.int32)
    st = stream if stream is not None else default_stream()
    _check(lib().fast_build_cst_batch(graph.handle, nq, arr, ctypes.byref(cfg) if cfg else None, st, outs,
                                      _p(status)))
    csts = []
    for i in range(nq):
        if status[i] != 0 or not outs[i]:
            csts.append(None)
            continue
        csts.append(Cst._adopt(graph, keep[2 * i], keep[2 * i + 1], _vp(outs[i]), st))
    return csts, status[:nq]


def partition_many(csts, cfg: Config | None = None, stream=None):
    """Partitions of many CSTs built together (fast_partition_batch): a list
    with a Chunks per CST, and the status array."""
    nq = len(csts)
    hs = (_vp * max(nq, 1))(*[c.handle if c is not None else None for c in csts])
    outs = (_vp * max(nq, 1))()
    status = np.zeros(max(nq, 1), np.int32)
    first = next((c for c in csts if c is not None), None)
    st = stream if stream is not None else (first.stream if first is not None else default_stream())
    _check(lib().fast_partition_batch(hs, nq, ctypes.byref(cfg) if cfg else None, st, outs, _p(status)))
    chunks = [Chunks._adopt(c, _vp(outs[i]), st) if status[i] == 0 and outs[i] else None for i, c in enumerate(csts)]
    return chunks, status[:nq]


class Batch:
    """Reusable batched matcher (fast_batch_*): one graph-replayed matcher
    launch per run for all queries."""

    def __init__(self, graph: Graph, max_queries: int, cfg: Config | None = None, threads: int = 0):
        h = _vp()
        _check(lib().fast_batch_create(graph.handle, ctypes.byref(cfg) if cfg else None, max_queries, threads,
                                       ctypes.byref(h)))
        self._h = h
        self.graph = graph

    def run(self, queries, stream=None):
        """queries: [(labels, edges)].  Returns (counts int64[n], status int32[n])."""
        arr, keep = _query_descs(queries)
        n = len(queries)
        counts = np.zeros(max(n, 1), np.uint64)
        status = np.zeros(max(n, 1), np.int32)
        _check(lib().fast_batch_run(self._h, n, arr, _p(counts), _p(status),
                                    stream if stream is not None else default_stream()))
        return counts[:n].astype(np.int64), status[:n]

    def timing(self):
        b, m, by, ch, fl = ctypes.c_double(), ctypes.c_double(), _u64(), _i64(), _u64()
        _check(lib().fast_batch_timing(self._h, ctypes.byref(b), ctypes.byref(m), ctypes.byref(by), ctypes.byref(ch)))
        _check(lib().fast_batch_bytes(self._h, None, ctypes.byref(fl)))
        return {"build_ms": b.value, "match_ms": m.value, "match_bytes": by.value, "floor_bytes": fl.value,
                "chunks": ch.value}

    def config(self, k: int, new: Config | None = None) -> Config:
        c = Config()
        _check(lib().fast_batch_config(self._h, k, ctypes.byref(c), ctypes.byref(new) if new else None))
        return new if new else c

    def autotune(self, sample, stream=None) -> float:
        arr, keep = _query_descs(sample)
        best = ctypes.c_double()
        _check(lib().fast_batch_autotune(self._h, len(sample), arr, ctypes.byref(best),
                                         stream if stream is not None else default_stream()))
        return best.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fast_free_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("count", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("t_arrive_ns", ctypes.c_uint64), ("t_start_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64)]


class Server:
    """Request loop with continuous batching over a resident graph
    (fast_server_*)."""

    def __init__(self, graph: Graph, budget_bytes: int, cfg: Config | None = None, workers: int = 0):
        h = _vp()
        _check(lib().fast_server_create(graph.handle, ctypes.byref(cfg) if cfg else None, int(budget_bytes),
                                        workers, ctypes.byref(h)))
        self._h = h
        self.graph = graph

    def submit(self, labels, edges) -> int:
        arr, keep = _query_descs([(labels, edges)])
        rid = _u64()
        _check(lib().fast_server_submit(self._h, ctypes.byref(arr[0]), ctypes.byref(rid)))
        return rid.value

    def poll(self, max_results: int = 1024, wait_ms: int = 0):
        out = (Result * max_results)()
        n = _i32()
        _check(lib().fast_server_poll(self._h, max_results, out, ctypes.byref(n), wait_ms))
        return [{"id": r.id, "count": r.count, "status": r.status, "t_arrive_ns": r.t_arrive_ns,
                 "t_start_ns": r.t_start_ns, "t_done_ns": r.t_done_ns} for r in out[:n.value]]

    def stats(self):
        p, r, b = _i64(), _i64(), _u64()
        _check(lib().fast_server_stats(self._h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(b)))
        return {"pending": p.value, "running": r.value, "in_use_bytes": b.value}

    def groups(self):
        """(groups formed, requests they held)."""
        gr, rq = _u64(), _u64()
        _check(lib().fast_server_groups(self._h, ctypes.byref(gr), ctypes.byref(rq)))
        return gr.value, rq.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fast_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def now_ns() -> int:
    return int(lib().fast_now_ns())


def match_batch(graph: Graph, queries, cfg: Config | None = None, stream=None):
    """fast_match_batch (one shot): (counts, status)."""
    arr, keep = _query_descs(queries)
    n = len(queries)
    counts = np.zeros(max(n, 1), np.uint64)
    status = np.zeros(max(n, 1), np.int32)
    _check(lib().fast_match_batch(graph.handle, n, arr, ctypes.byref(cfg) if cfg else None, _p(counts), _p(status),
                                  stream if stream is not None else default_stream()))
    return counts[:n].astype(np.int64), status[:n]


def match_noalloc(cst: Cst, chunks: Chunks | None = None, k: int = 0, emb_out=None, cfg: Config | None = None,
                  stream=None, check: bool = True):
    """fast_match_noalloc: the matcher with its scratch in a static device
    array, for callers that must not allocate.  emb_out (k > 0) must be a
    device buffer.  Returns dict(count, written, status)."""
    cnt, wr = _u64(), _u64()
    rc = lib().fast_match_noalloc(cst.handle, chunks.handle if chunks else None, ctypes.byref(cfg) if cfg else None,
                                  k, _p(emb_out), ctypes.byref(cnt), ctypes.byref(wr),
                                  stream if stream is not None else cst.stream)
    if check:
        _check(rc)
    return {"count": cnt.value, "written": wr.value, "status": rc}


def match_stats(cst: Cst, chunks: Chunks | None = None, cfg: Config | None = None, stream=None):
    """fast_match_stats: (algorithmic bytes, partial results per depth)."""
    out = np.zeros(cst.k + 1, np.uint64)
    _check(lib().fast_match_stats(cst.handle, chunks.handle if chunks else None, ctypes.byref(cfg) if cfg else None,
                                  _p(out), stream if stream is not None else cst.stream))
    return int(out[0]), out[1:].astype(np.int64)


def last_match_ms() -> float:
    """Event-timed duration of the last matcher kernel on this thread."""
    return float(lib().fast_last_match_ms())


def last_match_bytes() -> int:
    """Bytes the last fast_match on this thread requested."""
    return int(lib().fast_last_match_bytes())


def last_match_floor_bytes() -> int:
    """The floor of those bytes (fast_last_match_floor_bytes)."""
    return int(lib().fast_last_match_floor_bytes())


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().fast_kernel_launches())


def last_build_round_trips() -> int:
    """Host round trips of this thread's last batched CST build
    (fast_last_build_round_trips)."""
    return int(lib().fast_last_build_round_trips())
