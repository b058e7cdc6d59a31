"""fast_match_noalloc, the matcher entry point that allocates no device
memory, against fast_match on the same CST.

Some callers cannot allocate: an embedder whose GPU memory is all owned by
another allocator, a serving loop that must not enter the allocator once it
runs, code on a thread or callback that must not call into it.  For them the
matcher keeps its scratch in a static device array.  Its results must equal
those of the ordinary entry point -- exactly, since both are integer
enumerations -- on two calls in a row (the shared array keeps the previous
call's contents, so the second call also checks that they are cleared).

This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2102_10768_gb300 as F
import synth

pytestmark = pytest.mark.gpu


def _sorted(rows):
    rows = np.asarray(rows, dtype=np.int64)
    return rows[np.lexsort(rows.T[::-1])] if rows.shape[0] else rows


@pytest.fixture(scope="module")
def graphs():
    F.build()
    F.lib()
    w = synth.er_workload()
    er = F.Graph(w.n, w.edges, w.labels)
    rng = np.random.default_rng(11)
    n = 3000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(6000, 2)) if x[0] != x[1]]
    hub = F.Graph(n, np.array(e, np.int32), np.zeros(n, np.int32))
    return w, er, hub


def _compare(cst, chunks=None, cfg=None, kemb=None):
    import torch
    ref = F.match(cst, chunks, cfg=cfg)
    k = ref["count"] + 8 if kemb is None else kemb
    ref_rows = None
    if k:
        full = F.match(cst, chunks, k=k, cfg=cfg)
        ref_rows = full["emb"][:full["written"]]
    for _ in range(2):
        emb = torch.full((max(k, 1), cst.k), -1, dtype=torch.int32, device="cuda")
        r = F.match_noalloc(cst, chunks, k=k, emb_out=emb, cfg=cfg)
        assert r["count"] == ref["count"]
        if k:
            assert r["written"] == full["written"]
            got = emb[:r["written"]].cpu().numpy()
            if kemb is None:
                assert np.array_equal(_sorted(got), _sorted(ref_rows))
            else:
                assert len({tuple(x) for x in got.tolist()}) == got.shape[0]


def test_noalloc_equals_fast_match_er(graphs):
    w, er, _ = graphs
    for q in w.queries[:4]:
        cst = F.Cst(er, q.labels, q.edges)
        _compare(cst)
        _compare(cst, F.Chunks(cst, F.default_config(delta_w=max(1, cst.W // 16))))


def test_noalloc_equals_fast_match_skewed(graphs):
    _, _, hub = graphs
    cst = F.Cst(hub, np.zeros(4, np.int32), [[0, 1], [1, 2], [2, 3]])
    _compare(cst, kemb=0)
    _compare(cst, cfg=F.default_config(limit=100_000), kemb=4096)


def test_noalloc_rejects_host_buffer(graphs):
    w, er, _ = graphs
    q = w.queries[0]
    cst = F.Cst(er, q.labels, q.edges)
    with pytest.raises(F.FastError) as ei:
        F.match_noalloc(cst, k=4, emb_out=np.zeros((4, q.k), np.uint32))
    assert ei.value.code == F.FAST_ERR_INVALID
    assert F.lib().fast_match_noalloc_scratch_bytes() < 8 << 20
