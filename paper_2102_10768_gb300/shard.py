"""Sharding one query's CST chunks across ranks (one process per GPU).

The chunks of a partition are disjoint and complete search spaces (Sec. IV-B:
every embedding lies in exactly one chunk), so the ranks of a job can each
enumerate a subset of them and the query's count is the sum of the ranks'
counts -- the only exchange on the data path.  Every rank builds the same
CST and the same partition (both are deterministic), takes its share of the
chunks by the greedy rule below on their workload estimates W' (Sec. IV-C),
matches it, and the u64 counts are summed over the ranks.

Host logic only: the CUDA work is the library's (fast_chunks_select and the
matcher); the reduction goes through torch.distributed (NCCL on GPUs, gloo in
the CPU tests).
"""
from __future__ import annotations

import numpy as np


def assign_chunks(weights, world: int) -> list:
    """Greedy longest-processing-time split of chunks over `world` ranks:
    chunks in decreasing W' (ties to the smaller index) each go to the rank
    with the least W' so far (ties to the smaller rank).  Returns, per rank,
    its chunk indices in increasing order.  Every chunk goes to exactly one
    rank; the heaviest rank's total is at most the mean plus the largest W'."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.float64).reshape(-1)
    order = sorted(range(w.shape[0]), key=lambda i: (-w[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda x: (load[x], x))
        out[r].append(i)
        load[r] += float(w[i])
    return [np.array(sorted(x), dtype=np.int64) for x in out]


def allreduce_counts(counts, dist, device="cpu") -> np.ndarray:
    """Sum unsigned 64-bit counts over the ranks exactly: each count travels
    as its two 32-bit halves in int64 lanes (exact for up to 2^31 ranks), and
    the halves are recombined on the host.  Returns (sums, overflow): uint64
    sums, and per count whether its sum passed 2^64 - 1 (the sum then
    saturates there, as a count that reaches 2^64 in one launch does)."""
    import torch
    c = np.asarray(counts, dtype=np.uint64).reshape(-1)
    lo = (c & np.uint64(0xFFFFFFFF)).astype(np.int64)
    hi = (c >> np.uint64(32)).astype(np.int64)
    t = torch.from_numpy(np.concatenate([lo, hi])).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    s = t.cpu().numpy()
    n = c.shape[0]
    lo_s = s[:n].astype(object)
    hi_s = s[n:].astype(object)
    out = np.zeros(n, dtype=np.uint64)
    over = np.zeros(n, dtype=bool)
    for i in range(n):
        v = int(hi_s[i]) * (1 << 32) + int(lo_s[i])
        if v >= 1 << 64:
            over[i] = True
            v = (1 << 64) - 1
        out[i] = np.uint64(v)
    return out, over
