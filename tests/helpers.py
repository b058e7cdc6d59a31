"""Shared helpers for the parity tests: compare the CUDA path (through the
C ABI binding) with the oracle on the same seeded inputs."""
import numpy as np

import oracle


def gpu_tree_global(cst, u):
    """GPU tree lists into u with data-vertex ids."""
    off, idx = cst.tree_lists(u)
    cu = cst.candidates(u)
    return off, cu[idx.astype(np.int64)] if idx.size else idx.astype(np.int32)


def compare_cst(gcst, ocst, k):
    """Exact equality of root, t_q, order, candidate sets, tree lists,
    non-tree lists and the workload estimate."""
    assert gcst.root == ocst.root
    assert gcst.parent.tolist() == ocst.parent.tolist()
    assert gcst.order.tolist() == ocst.order.tolist()
    for u in range(k):
        assert np.array_equal(gcst.candidates(u), ocst.cand(u)), f"C({u}) differs"
    for u in range(k):
        if ocst.parent[u] < 0:
            continue
        goff, gvals = gpu_tree_global(gcst, u)
        ooff, ovals = ocst.tree(u)
        assert np.array_equal(goff, ooff), f"tree offsets into {u} differ"
        assert np.array_equal(gvals, ovals), f"tree lists into {u} differ"
    gnt = {(a, b): (off, idx) for a, b, off, idx in gcst.nontree()}
    ont = {(a, b): (off, vals) for a, b, off, vals in ocst.nontree()}
    assert set(gnt) == set(ont)
    for key, (ooff, ovals) in ont.items():
        goff, gidx = gnt[key]
        cb = gcst.candidates(key[1])
        assert np.array_equal(goff, ooff)
        assert np.array_equal(cb[gidx.astype(np.int64)] if gidx.size else gidx.astype(np.int32), ovals)
    wf, wi, _, _ = ocst.workload()
    assert gcst.W == wi
    assert abs(gcst.Wf - wf) <= 1e-9 * max(1.0, abs(wf))
    for u in range(k):
        _, _, _, ci = ocst.workload(dump_u=u)
        assert np.array_equal(gcst.workload(u), ci.astype(np.uint64)), f"c_{u} differs"


def gpu_chunks_global(gcst, chunks):
    """GPU chunk descriptors with data-vertex ids in the prefix."""
    out = []
    cands = {}
    for (j, pre, a, b, w, i) in chunks.copy():
        g = []
        for p, m in enumerate(pre):
            u = int(gcst.order[p])
            if u not in cands:
                cands[u] = gcst.candidates(u)
            g.append(int(cands[u][m]))
        out.append((j, tuple(g), a, b, w, i))
    return out


def sorted_rows(a):
    a = np.asarray(a)
    if a.shape[0] == 0:
        return a
    return a[np.lexsort(a.T[::-1])]


def csr_by_label(off, col, labels):
    """The CSR's rows reordered by (label of the neighbour, neighbour id): the
    library's layout when its ids and labels fit one 64-bit sort key."""
    off = np.asarray(off, np.int64)
    col = np.asarray(col)
    labels = np.asarray(labels)
    row = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    order = np.lexsort((col, labels[col], row))
    return off, col[order]
