"""Pins for the seeded input generators (CPU).

The generators feed both the CUDA path and the oracle, so a mistake here
would go unseen by the parity tests: both sides would agree on the wrong
input.  These tests check each generator against what its model fixes:
edge sets are simple graphs of exactly m edges, degrees follow the model's
closed form, label frequencies follow their distribution, and a random-walk
query is connected, labelled from G and matched by the walk itself.
"""
import numpy as np
import pytest

import oracle
import synth


def _pairs(e):
    lo = np.minimum(e[:, 0], e[:, 1]).astype(np.int64)
    hi = np.maximum(e[:, 0], e[:, 1]).astype(np.int64)
    return (lo << 32) | hi


def _assert_simple(e, n, m):
    assert e.shape == (m, 2) and e.dtype == np.int32
    assert e.min() >= 0 and e.max() < n
    assert not np.any(e[:, 0] == e[:, 1]), "self-loop"
    assert np.unique(_pairs(e)).shape[0] == m, "repeated edge"


def _degree(e, n):
    return np.bincount(e.ravel(), minlength=n)


# --------------------------------------------------------------- edges

def test_er_edges_simple_and_binomial():
    n, m = 4000, 40_000
    e = synth.er_edges(n, m, 11)
    _assert_simple(e, n, m)
    d = _degree(e, n)
    assert d.sum() == 2 * m
    # G(n, m): a degree is close to Binomial(n-1, 2m/(n(n-1))), variance ~ mean
    ratio = d.var() / d.mean()
    assert 0.85 < ratio < 1.15, ratio


def test_er_edges_complete_graph():
    # m = n(n-1)/2 forces every pair exactly once
    n = 40
    e = synth.er_edges(n, n * (n - 1) // 2, 3)
    _assert_simple(e, n, n * (n - 1) // 2)
    assert np.all(_degree(e, n) == n - 1)


def test_er_edges_rejects_too_many():
    with pytest.raises(RuntimeError):
        synth.er_edges(10, 46, 1)


def test_edges_deterministic_and_seeded():
    a = synth.er_edges(1000, 5000, 7)
    b = synth.er_edges(1000, 5000, 7)
    c = synth.er_edges(1000, 5000, 8)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    a = synth.chung_lu_edges(1000, 5000, 2.1, 7)
    assert np.array_equal(a, synth.chung_lu_edges(1000, 5000, 2.1, 7))
    a = synth.rmat_edges(10, 5000, 7)
    assert np.array_equal(a, synth.rmat_edges(10, 5000, 7))


def test_chung_lu_degree_follows_weight():
    # Each draw picks both endpoints with probability p_i = w_i / sum(w),
    # w_i = (i+1)^(-1/(gamma-1)); draws repeat until m distinct non-loop pairs
    # are kept.  After D draws, pair {i, j} is present with probability
    # 1 - (1 - 2 p_i p_j)^D, D fixed by the expected number of present pairs
    # being m.  The expected degree of i is the sum over j of that probability.
    # Band means of the measured degrees match it.
    n, m, gamma = 2000, 20_000, 2.1
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    p = w / w.sum()
    lq = np.log1p(-2.0 * np.outer(p, p))
    np.fill_diagonal(lq, 0.0)
    lo, hi = float(m), 4.0 * m
    for _ in range(32):
        mid = 0.5 * (lo + hi)
        if (1.0 - np.exp(mid * lq)).sum() / 2 < m:
            lo = mid
        else:
            hi = mid
    want = (1.0 - np.exp(0.5 * (lo + hi) * lq)).sum(axis=1)
    e = synth.chung_lu_edges(n, m, gamma, 5)
    _assert_simple(e, n, m)
    d = _degree(e, n).astype(np.float64)
    for a, b in ((0, 10), (10, 50), (50, 200), (200, 800), (800, n)):
        r = d[a:b].mean() / want[a:b].mean()
        assert abs(r - 1.0) < 0.04, (a, b, r)
    # heavy head
    assert d[:10].mean() > 20 * d.mean()


def test_rmat_degree_skew_and_uniform_special_case():
    scale, m = 13, 60_000
    n = 1 << scale
    e = synth.rmat_edges(scale, m, 9)
    _assert_simple(e, n, m)
    d = _degree(e, n)
    assert d.max() > 20 * d.mean()
    # a = b = c = d = 1/4: every bit of both endpoints is a fair coin, so the
    # endpoints are uniform and the graph is G(n, m)-like
    u = synth.rmat_edges(scale, m, 9, a=0.25, b=0.25, c=0.25)
    _assert_simple(u, n, m)
    du = _degree(u, n)
    ratio = du.var() / du.mean()
    assert 0.85 < ratio < 1.15, ratio
    assert du.max() < 4 * du.mean()


# -------------------------------------------------------------- labels

def _chi2_ok(counts, p, z=6.0):
    """Every frequency within z standard deviations of its expectation."""
    n = counts.sum()
    exp = n * p
    sd = np.sqrt(n * p * (1 - p))
    return np.all(np.abs(counts - exp) <= z * sd)


def test_labels_uniform():
    n, L = 200_000, 12
    lab = synth.labels_uniform(n, L, 4)
    assert lab.dtype == np.int32 and lab.min() >= 0 and lab.max() < L
    assert _chi2_ok(np.bincount(lab, minlength=L), np.full(L, 1.0 / L))
    assert np.array_equal(lab, synth.labels_uniform(n, L, 4))


def test_labels_zipf():
    n, L = 200_000, 16
    lab = synth.labels_zipf(n, L, 4)
    assert lab.min() >= 0 and lab.max() < L
    c = np.bincount(lab, minlength=L)
    p = 1.0 / np.arange(1, L + 1)
    p /= p.sum()
    assert _chi2_ok(c, p)
    assert np.all(np.diff(c[:4]) < 0), c      # label 0 the most frequent
    # s = 0 reduces Zipf to the uniform distribution
    u = synth.labels_zipf(n, L, 4, s=0.0)
    assert _chi2_ok(np.bincount(u, minlength=L), np.full(L, 1.0 / L))


def test_labels_single_label():
    assert np.all(synth.labels_uniform(100, 1, 1) == 0)
    assert np.all(synth.labels_zipf(100, 1, 1) == 0)


# ---------------------------------------------------- walk queries

def _connected(k, qe):
    adj = [[] for _ in range(k)]
    for a, b in qe:
        adj[a].append(b)
        adj[b].append(a)
    seen, stack = {0}, [0]
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return len(seen) == k


@pytest.fixture(scope="module")
def walk_setup():
    n, m, L = 20_000, 200_000, 8
    e = synth.chung_lu_edges(n, m, 2.1, 21)
    lab = synth.labels_zipf(n, L, 21)
    pairs = set(_pairs(e).tolist())
    wg = synth.WalkGraph(n, e)
    og = oracle.Graph(n, e, lab)
    yield n, e, lab, pairs, wg, og
    wg.close()
    og.close()


@pytest.mark.parametrize("kind,k", [("induced", 2), ("induced", 4), ("induced", 8), ("sparse", 2),
                                    ("sparse", 4), ("sparse", 8), ("sparse", 16),
                                    ("dense", 8), ("dense", 16)])
def test_walk_query_properties(walk_setup, kind, k):
    n, e, lab, pairs, wg, og = walk_setup
    for stream in range(6):
        q = wg.query(lab, k, kind, 77, stream)
        v = q.verts
        assert q.k == k and v.shape == (k,)
        assert np.unique(v).shape[0] == k and v.min() >= 0 and v.max() < n
        assert np.array_equal(q.labels, lab[v])
        qe = q.edges
        assert qe.shape[1] == 2 and qe.min() >= 0 and qe.max() < k
        assert not np.any(qe[:, 0] == qe[:, 1])
        assert np.unique(_pairs(qe)).shape[0] == qe.shape[0]
        # every query edge is an edge of G between the walk's vertices
        got = {(int(min(a, b)), int(max(a, b))) for a, b in qe}
        induced = {(i, j) for i in range(k) for j in range(i + 1, k)
                   if ((int(min(v[i], v[j])) << 32) | int(max(v[i], v[j]))) in pairs}
        assert got <= induced
        assert _connected(k, qe.tolist())
        if kind in ("induced", "dense"):
            assert got == induced
        if kind == "dense":
            assert q.avg_degree > 3.0
        if kind == "sparse":
            assert k - 1 <= qe.shape[0] <= max(k - 1, (3 * k) // 2)
        # the walk itself is an embedding of the query (Definition 1)
        assert oracle.invalid_rows(og, q.labels, qe, v[None, :]) == 0


def test_walk_query_deterministic(walk_setup):
    _, _, lab, _, wg, _ = walk_setup
    a = wg.query(lab, 8, "sparse", 5, 3)
    b = wg.query(lab, 8, "sparse", 5, 3)
    c = wg.query(lab, 8, "sparse", 5, 4)
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.edges, b.edges)
    assert not np.array_equal(a.verts, c.verts)


def test_dense_query_impossible_below_five_vertices(walk_setup):
    # average degree above 3 needs more than 3k/2 edges, and k <= 4 vertices
    # have at most k(k-1)/2 <= 3k/2 pairs
    _, _, lab, _, wg, _ = walk_setup
    with pytest.raises(RuntimeError):
        wg.query(lab, 4, "dense", 1, 0, max_attempts=50)


def test_walk_query_isolated_graph_fails():
    # no edges: no walk can reach k > 1 vertices
    wg = synth.WalkGraph(10, np.zeros((0, 2), np.int32))
    try:
        with pytest.raises(RuntimeError):
            wg.query(np.zeros(10, np.int32), 3, "induced", 1, 0, max_attempts=5)
        q = wg.query(np.zeros(10, np.int32), 1, "induced", 1, 0)
        assert q.k == 1 and q.edges.shape[0] == 0
    finally:
        wg.close()


# ------------------------------------- bit-exact restatement, tiny inputs
#
# The generators draw every number as a pure function of (seed, stream,
# counter) through the splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).
# Below, that finaliser is written out in Python and pinned to the published
# splitmix64 output sequence; each generator's recipe is then restated on top
# of it and compared with the C output element by element.

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z):
    z = (z + _GOLDEN) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _rkey(seed, stream):
    return _mix64(_mix64(seed) ^ ((stream * 0xD1B54A32D192ED03) & _M64))


def _rnd(key, ctr):
    return _mix64((key + ctr * _GOLDEN) & _M64)


def _below(r, n):
    return (r * n) >> 64


def _u01(r):
    return (r >> 11) * (1.0 / 9007199254740992.0)


def test_splitmix64_published_sequence():
    # splitmix64 seeded with state 0: the state advances by the golden-ratio
    # increment and each output is the finaliser of the new state
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [_mix64((i * _GOLDEN) & _M64) for i in range(3)] == want


def _first_unique(draw, m):
    out, seen, ctr = [], set(), 0
    while len(out) < m:
        s, d = draw(ctr)
        ctr += 1
        key = (min(s, d), max(s, d))
        if s != d and key not in seen:
            seen.add(key)
            out.append((s, d))
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def _cdf_pick(cdf, x):
    for i, c in enumerate(cdf):
        if c > x:
            return i
    return len(cdf) - 1


def test_er_edges_bit_exact():
    n, m, seed = 37, 120, 12345
    key = _rkey(seed, 1)
    want = _first_unique(lambda c: (_below(_rnd(key, 2 * c), n), _below(_rnd(key, 2 * c + 1), n)), m)
    assert np.array_equal(synth.er_edges(n, m, seed), want)


def test_chung_lu_edges_bit_exact():
    n, m, gamma, seed = 60, 150, 2.1, 99
    w = [float(i + 1) ** (-1.0 / (gamma - 1.0)) for i in range(n)]
    acc, cdf = 0.0, []
    for x in w:
        acc += x
        cdf.append(acc)
    cdf = [c / acc for c in cdf]
    cdf[-1] = 2.0
    key = _rkey(seed, 2)
    want = _first_unique(lambda c: (_cdf_pick(cdf, _u01(_rnd(key, 2 * c))),
                                    _cdf_pick(cdf, _u01(_rnd(key, 2 * c + 1)))), m)
    assert np.array_equal(synth.chung_lu_edges(n, m, gamma, seed), want)


def test_rmat_edges_bit_exact():
    scale, m, seed, a, b, c = 6, 200, 4242, 0.57, 0.19, 0.19
    n = 1 << scale
    perm = list(range(n))
    pk = _rkey(seed, 4)
    for i in range(n - 1, 0, -1):           # Fisher-Yates
        j = _below(_rnd(pk, i), i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    key = _rkey(seed, 3)

    def draw(ctr):
        s = d = 0
        for lev in range(scale):
            r = _u01(_rnd(key, ctr * 64 + lev))
            bs, bd = (0, 0) if r < a else (0, 1) if r < a + b else (1, 0) if r < a + b + c else (1, 1)
            s, d = (s << 1) | bs, (d << 1) | bd
        return perm[s], perm[d]

    want = _first_unique(draw, m)
    assert np.array_equal(synth.rmat_edges(scale, m, seed, a, b, c), want)


def test_labels_bit_exact():
    n, L, seed = 500, 7, 31337
    k5 = _rkey(seed, 5)
    want = [_below(_rnd(k5, i), L) for i in range(n)]
    assert synth.labels_uniform(n, L, seed).tolist() == want
    s = 1.0
    acc, cdf = 0.0, []
    for i in range(L):
        acc += float(i + 1) ** (-s)
        cdf.append(acc)
    cdf = [c / acc for c in cdf]
    cdf[-1] = 2.0
    k6 = _rkey(seed, 6)
    want = [_cdf_pick(cdf, _u01(_rnd(k6, i))) for i in range(n)]
    assert synth.labels_zipf(n, L, seed, s).tolist() == want


def test_generators_do_not_depend_on_the_thread_count():
    """The edge lists (and the walks, whose graph is sorted the same way) come
    out the same with 1 and with 3 OpenMP threads, on inputs large enough for
    the sort to split its ranges across threads."""
    import os
    import subprocess
    import sys
    code = (
        "import hashlib, numpy as np, synth\n"
        "h = lambda a: hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest()\n"
        "e = synth.chung_lu_edges(200_000, 1_200_000, 2.1, 3)\n"
        "r = synth.rmat_edges(17, 900_000, 3)\n"
        "w = synth.WalkGraph(200_000, e).query(synth.labels_zipf(200_000, 8, 3), 8, 'sparse', 3, 1)\n"
        "print(h(e), h(r), h(w.verts), h(w.edges))\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t, PYTHONPATH=root)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True, timeout=300).stdout)
    assert outs[0] == outs[1] and outs[0].strip()
