"""fast_match_noalloc, the matcher entry point that allocates no device
memory, against fast_match on the same CST and against the oracle.

Some callers cannot allocate: an embedder whose GPU memory is all owned by
another allocator, a serving loop that must not enter the allocator once it
runs, code on a thread or callback that must not call into it.  For them the
matcher keeps its scratch in a static device array.  Its results must equal
those of the ordinary entry point and the oracle's -- exactly, since both are
integer enumerations -- on two calls in a row (the shared array keeps the
previous call's contents, so the second call also checks that they are
cleared).  Each call runs with an allocation failure armed on the library's
host-side failure hook: a call that reached any device allocation would fail
with FAST_ERR_OOM, and the hook's countdown would have moved.

This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
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
    oer = oracle.Graph(w.n, w.edges, w.labels)
    rng = np.random.default_rng(11)
    n = 3000
    e = [(0, v) for v in range(1, n)] + [tuple(x) for x in rng.integers(1, n, size=(6000, 2)) if x[0] != x[1]]
    e = np.array(e, np.int32)
    hub = F.Graph(n, e, np.zeros(n, np.int32))
    ohub = oracle.Graph(n, e, np.zeros(n, np.int32))
    return w, er, oer, hub, ohub


def _noalloc(cst, chunks, k, emb, cfg):
    """One fast_match_noalloc call with the next device allocation armed to
    fail; checks that the call returned FAST_OK without reaching it."""
    F.inject_alloc_failure(0)
    try:
        r = F.match_noalloc(cst, chunks, k=k, emb_out=emb, cfg=cfg)
    finally:
        left = F.inject_alloc_failure(-1)
    assert left == 0, "fast_match_noalloc reached a device allocation"
    assert r["status"] == F.FAST_OK
    return r


def _compare(cst, want, chunks=None, cfg=None, kemb=None):
    """fast_match_noalloc twice in a row: counts equal fast_match's and the
    oracle's `want` (count, sorted rows or None); rows equal as sets when
    every embedding is written, else distinct and among fast_match's set."""
    import torch
    ref = F.match(cst, chunks, cfg=cfg)
    assert ref["count"] == want[0]
    k = ref["count"] + 8 if kemb is None else kemb
    if k:
        full = F.match(cst, chunks, k=k, cfg=cfg)
        ref_rows = full["emb"][:full["written"]]
    for _ in range(2):
        emb = torch.full((max(k, 1), cst.k), -1, dtype=torch.int32, device="cuda")
        r = _noalloc(cst, chunks, k, emb, cfg)
        assert r["count"] == ref["count"] == want[0]
        if k:
            assert r["written"] == full["written"]
            got = emb[:r["written"]].cpu().numpy()
            if kemb is None:
                assert np.array_equal(_sorted(got), _sorted(ref_rows))
                assert np.array_equal(_sorted(got), _sorted(want[1]))
            else:
                assert len({tuple(x) for x in got.tolist()}) == got.shape[0]


def test_noalloc_equals_fast_match_and_oracle_er(graphs):
    w, er, oer, _, _ = graphs
    for q in w.queries[:4]:
        o = oracle.match(oer, q.labels, q.edges, max_emb=1 << 20)
        assert o["complete"]
        want = (o["count"], o["emb"])
        cst = F.Cst(er, q.labels, q.edges)
        _compare(cst, want)
        _compare(cst, want, F.Chunks(cst, F.default_config(delta_w=max(1, cst.W // 16))))


def test_noalloc_equals_fast_match_and_oracle_skewed(graphs):
    _, _, _, hub, ohub = graphs
    ql, qe = np.zeros(4, np.int32), [[0, 1], [1, 2], [2, 3]]
    cst = F.Cst(hub, ql, qe)
    _compare(cst, (oracle.count(ohub, ql, qe), None), kemb=0)
    _compare(cst, (oracle.match(ohub, ql, qe, limit=100_000)["count"], None),
             cfg=F.default_config(limit=100_000), kemb=4096)


def test_noalloc_rejects_host_buffer(graphs):
    w, er, _, _, _ = graphs
    q = w.queries[0]
    cst = F.Cst(er, q.labels, q.edges)
    with pytest.raises(F.FastError) as ei:
        F.match_noalloc(cst, k=4, emb_out=np.zeros((4, q.k), np.uint32))
    assert ei.value.code == F.FAST_ERR_INVALID
    assert F.lib().fast_match_noalloc_scratch_bytes() < 8 << 20


def test_noalloc_rejects_more_root_runs_than_its_scratch_holds():
    # a path over 40,000 vertices and a one-edge query: every vertex is a root
    # candidate, and 8 CTAs of 8 warps per SM ask for 4 runs per warp, more
    # than the static scratch's 32768 descriptors on any GPU of 128 SMs or more
    import torch
    n = 40_000
    if torch.cuda.get_device_properties(0).multi_processor_count * 8 * 8 * 4 <= 32768:
        pytest.skip("too few SMs to pass the limit with this launch shape")
    e = np.stack([np.arange(n - 1), np.arange(1, n)], 1).astype(np.int32)
    g = F.Graph(n, e, np.zeros(n, np.int32))
    cst = F.Cst(g, np.zeros(2, np.int32), [[0, 1]])
    with pytest.raises(F.FastError) as ei:
        F.match_noalloc(cst, cfg=F.default_config(warps_per_block=8, blocks_per_sm=8))
    assert ei.value.code == F.FAST_ERR_INVALID
    assert "root runs" in str(ei.value)
    # within the limit the same call counts every ordered edge
    r = F.match_noalloc(cst, cfg=F.default_config(warps_per_block=8, blocks_per_sm=4))
    assert r["count"] == 2 * (n - 1)
