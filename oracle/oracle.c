/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU restatement of what the subgraph-matching path computes.
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline may load it; the CUDA library never does, and the two share no
 * code.
 *
 * Contents
 *   1. Data graph: symmetrised, loop-free, duplicate-free adjacency with sorted
 *      neighbour lists (the paper studies simple undirected graphs, Sec. II-A).
 *   2. oracle_match: the problem statement of Sec. II-A -- every injective map
 *      M: V(q) -> V(G) with l_q(u) = l_G(M(u)) and (M(u), M(u')) in E(G) for
 *      every query edge (Definition 1) -- found by plain backtracking over G
 *      with no auxiliary structure.  Optional per-query-vertex allowed sets
 *      restrict M(u) (used to count one partition of the search space, and to
 *      count the partial results that a search over the candidate search
 *      tree must extend).
 *   3. CST restatement (Algorithm 1, Sec. IV-A), the workload estimate
 *      (Sec. IV-C) and the partition of Algorithm 2 live in cst_ref.c.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;
    int64_t* off;      /* [n+1] */
    int32_t* adj;      /* [off[n]] sorted, unique, no self loops */
    int32_t* lab;      /* [n] */
} og;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

og* oracle_graph_new(int64_t n, int64_t m, const int32_t* edges, const int32_t* labels) {
    og* g = (og*)calloc(1, sizeof(og));
    if (!g) return NULL;
    g->n = n;
    g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->lab = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->off || !g->lab || !deg) return NULL;
    memcpy(g->lab, labels, (size_t)n * sizeof(int32_t));
    for (int64_t e = 0; e < m; e++) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n) { free(deg); return NULL; }
        if (a == b) continue;
        deg[a]++; deg[b]++;
    }
    int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    pos[0] = 0;
    for (int64_t v = 0; v < n; v++) pos[v + 1] = pos[v] + deg[v];
    int32_t* raw = (int32_t*)malloc((size_t)(pos[n] > 0 ? pos[n] : 1) * sizeof(int32_t));
    int64_t* cur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    memcpy(cur, pos, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; e++) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a == b) continue;
        raw[cur[a]++] = b; raw[cur[b]++] = a;
    }
    /* sort each list, drop repeats */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; v++) {
        int64_t s = pos[v], e = pos[v + 1];
        qsort(raw + s, (size_t)(e - s), sizeof(int32_t), cmp_i32);
        int64_t w = s;
        for (int64_t i = s; i < e; i++)
            if (i == s || raw[i] != raw[i - 1]) raw[w++] = raw[i];
        deg[v] = w - s;
    }
    for (int64_t v = 0; v < n; v++) g->off[v + 1] = g->off[v] + deg[v];
    g->adj = (int32_t*)malloc((size_t)(g->off[n] > 0 ? g->off[n] : 1) * sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; v++)
        memcpy(g->adj + g->off[v], raw + pos[v], (size_t)deg[v] * sizeof(int32_t));
    free(raw); free(cur); free(pos); free(deg);
    return g;
}

void oracle_graph_free(og* g) {
    if (!g) return;
    free(g->off); free(g->adj); free(g->lab); free(g);
}

int64_t oracle_graph_nadj(const og* g) { return g->off[g->n]; }

void oracle_graph_csr(const og* g, int64_t* off, int32_t* adj) {
    memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(adj, g->adj, (size_t)g->off[g->n] * sizeof(int32_t));
}

/* (a, b) in E(G), by binary search in a's sorted list */
static int has_edge(const og* g, int32_t a, int32_t b) {
    int64_t lo = g->off[a], hi = g->off[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (g->adj[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < g->off[a + 1] && g->adj[lo] == b;
}

static int in_sorted(const int32_t* a, int64_t n, int32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == x;
}

/* ------------------------------------------------------------ search */

#define OMAXK 64

typedef struct {
    const og* g;
    int k;
    const int32_t* ql;
    int order[OMAXK];          /* position -> query vertex */
    int par[OMAXK];            /* position -> position of the vertex we extend from */
    int nb[OMAXK];             /* number of other earlier neighbours */
    int bn[OMAXK][OMAXK];      /* their positions */
    const int64_t* aoff;       /* allowed sets, per query vertex */
    const int32_t* av;
    const uint8_t* aon;
    int64_t max_emb;
    int32_t* emb;
    int64_t* emb_slot;         /* shared slot counter */
    int64_t budget;
    uint64_t limit;            /* stop once this many embeddings are found (0: none) */
    uint64_t* found;           /* shared count towards the limit */
} sctx;

typedef struct {
    uint64_t count;
    uint64_t depth[OMAXK];     /* valid partial results with d+1 positions mapped */
    double balg[2];            /* bytes to extend them: floor and ceiling (see oracle_match) */
    int64_t nodes;
    int over;
} sacc;

static int allowed(const sctx* c, int u, int32_t v) {
    if (!c->aon || !c->aon[u]) return 1;
    return in_sorted(c->av + c->aoff[u], c->aoff[u + 1] - c->aoff[u], v);
}

/* The CST list of x towards u when the allowed sets are the tree's
 * candidate sets: { w in N_G(x) : l(w) = l_q(u), w allowed for u }, in
 * increasing id (N_G(x) is sorted).  Returns its length; fills buf. */
static int64_t cst_list(const sctx* c, int32_t x, int u, int32_t* buf) {
    const og* g = c->g;
    int64_t n = 0;
    for (int64_t i = g->off[x]; i < g->off[x + 1]; i++) {
        int32_t w = g->adj[i];
        if (g->lab[w] == c->ql[u] && allowed(c, u, w)) buf[n++] = w;
    }
    return n;
}

/* Bytes a search over the candidate search tree reads to extend the valid
 * partial M[0..d) to position d.  The candidates of position d are the
 * intersection of the CST list from the image of its tree parent and the
 * lists from the images of its earlier non-tree neighbours (Alg. 5 and 7;
 * the CST lists, with the allowed sets taken as the candidate sets).
 *
 * lo[0], the floor: what a search that scans the shortest of those lists
 * (the generator) and checks its entries against the others must read --
 * 4 B for the image of the last mapped position, 16 B of offsets (begin and
 * end) per list, 4 B per generator entry, and 4 B for the data vertex of
 * each entry in every list while an earlier position has the same label
 * (the visited check, Alg. 6).
 *
 * lo[1], a ceiling for a warp that takes the generator 32 entries at a time
 * (S = ceil(|G| / 32) segments) and tests them against each other list L by
 * a merge with a forward-only cursor: tiles of 32 entries whose positions
 * never decrease except for one re-read at each segment start (at most
 * |L| + 32 S entries), and per tile that holds no pending candidate one
 * galloping search (one round of 32 probes, then at most five 33-way
 * refinement rounds of 32 probes, since a gallop spans at most 32 * 2^25
 * entries), at most min(|G|, ceil(|L| / 32) + S) of them.  lo[1] = lo[0] +
 * sum over L of 4 (|L| + 32 S) + 4 * 32 * 6 * min(|G|, ceil(|L|/32) + S). */
static void extension_bytes(const sctx* c, const int32_t* M, int d, double* lo) {
    const og* g = c->g;
    const int u = c->order[d];
    const int nl = 1 + c->nb[d];                    /* the tree list, then the non-tree lists */
    int32_t* L[OMAXK];
    int64_t len[OMAXK];
    for (int j = 0; j < nl; j++) {
        const int32_t x = j == 0 ? M[c->par[d]] : M[c->bn[d][j - 1]];
        const int64_t deg = g->off[x + 1] - g->off[x];
        L[j] = (int32_t*)malloc((size_t)(deg > 0 ? deg : 1) * sizeof(int32_t));
        len[j] = cst_list(c, x, u, L[j]);
    }
    int gi = 0;                                     /* the generator: shortest, ties to the earlier list */
    for (int j = 1; j < nl; j++) if (len[j] < len[gi]) gi = j;
    const int64_t ng = len[gi];
    int same = 0;
    for (int j = 0; j < d; j++) if (c->ql[c->order[j]] == c->ql[u]) same = 1;
    int64_t inter = 0;                              /* generator entries present in every list */
    for (int64_t i = 0; i < ng; i++) {
        int in_all = 1;
        for (int j = 0; j < nl && in_all; j++)
            if (j != gi && !in_sorted(L[j], len[j], L[gi][i])) in_all = 0;
        inter += in_all;
    }
    double b = 4.0 + 16.0 * nl + 4.0 * (double)ng + (same ? 4.0 * (double)inter : 0.0);
    double extra = 0.0;
    const int64_t segs = (ng + 31) / 32;
    for (int j = 0; j < nl; j++) {
        if (j == gi || ng == 0) continue;
        int64_t gallops = (len[j] + 31) / 32 + segs;
        if (gallops > ng) gallops = ng;
        extra += 4.0 * (double)(len[j] + 32 * segs) + 4.0 * 32.0 * 6.0 * (double)gallops;
    }
    for (int j = 0; j < nl; j++) free(L[j]);
    lo[0] += b;
    lo[1] += b + extra;
}

static void emit(const sctx* c, const int32_t* M) {
    if (!c->emb || c->max_emb <= 0) return;
    int64_t s = __atomic_fetch_add(c->emb_slot, 1, __ATOMIC_RELAXED);
    if (s >= c->max_emb) return;
    for (int i = 0; i < c->k; i++) c->emb[s * c->k + c->order[i]] = M[i];
}

static void extend(const sctx* c, sacc* a, int32_t* M, int d, int want_balg) {
    /* M[0..d) maps positions 0..d-1 and is a valid partial embedding */
    a->depth[d - 1]++;
    if (d == c->k) {
        if (c->limit) {
            uint64_t f = __atomic_fetch_add(c->found, 1, __ATOMIC_RELAXED);
            if (f >= c->limit) { a->over = 2; return; }
        }
        a->count++;
        emit(c, M);
        return;
    }
    if (a->over) return;
    if (c->limit && __atomic_load_n(c->found, __ATOMIC_RELAXED) >= c->limit) { a->over = 2; return; }
    const og* g = c->g;
    int u = c->order[d];
    int32_t x = M[c->par[d]];
    a->nodes += 1 + (g->off[x + 1] - g->off[x]);
    if (c->budget > 0 && a->nodes > c->budget) { a->over = 1; return; }
    if (want_balg) extension_bytes(c, M, d, a->balg);
    /* candidates: N_G(x), or the allowed set of u when that is shorter
     * (then adjacency to x is tested by binary search) */
    int64_t na = (c->aon && c->aon[u]) ? c->aoff[u + 1] - c->aoff[u] : -1;
    int from_allow = na >= 0 && na < g->off[x + 1] - g->off[x];
    int64_t lo = from_allow ? c->aoff[u] : g->off[x];
    int64_t hi = from_allow ? c->aoff[u + 1] : g->off[x + 1];
    for (int64_t i = lo; i < hi; i++) {
        int32_t v = from_allow ? c->av[i] : g->adj[i];
        if (g->lab[v] != c->ql[u]) continue;
        if (from_allow && !has_edge(g, x, v)) continue;
        int ok = 1;
        for (int j = 0; j < d && ok; j++) if (M[j] == v) ok = 0;          /* injective */
        for (int j = 0; j < c->nb[d] && ok; j++)
            if (!has_edge(g, M[c->bn[d][j]], v)) ok = 0;                     /* edges */
        if (!ok || (!from_allow && !allowed(c, u, v))) continue;
        M[d] = v;
        extend(c, a, M, d + 1, want_balg);
        if (a->over) return;
    }
}

/*
 * Enumerate all embeddings of q in G (Definition 1).
 *
 * q: k vertices with labels ql[k], nqe undirected edges qe[nqe][2].
 * order: position -> query vertex (NULL: breadth-first from query vertex 0,
 *        neighbours in increasing id).  Every position after the first must
 *        have an earlier neighbour; par[] (NULL: the earliest such neighbour)
 *        names the position whose image's neighbours are scanned.
 * allow_on[u] != 0 restricts M(u) to the sorted set
 *        allow_v[allow_off[u] .. allow_off[u+1]).
 * Outputs: *count_out = number of embeddings; up to max_emb of them in
 *        emb_out[max_emb][k] indexed by query vertex id (any order);
 *        depth_out[d] (nullable) = number of partial embeddings of the first
 *        d+1 positions that satisfy labels, injectivity, every edge among
 *        them and the allowed sets; *balg_out (nullable) = the bytes a search
 *        over the candidate search tree requests to extend every such partial
 *        embedding of d = 1..k-1 positions (extension_bytes): balg_out[0]
 *        the floor, balg_out[1] the ceiling, with the allowed sets taken as
 *        the tree's candidate sets.
 * limit (> 0) stops the search once `limit` embeddings are found; the count
 * is then exactly min(total, limit) and the rows any such embeddings.
 * Returns 0, 1 when some thread exceeded node_budget (>0) work units (one
 * per extended partial result plus one per neighbour scanned; the budget is
 * per thread; counts are then partial), or a negative code on invalid input.
 */
int oracle_match(const og* g, int k, const int32_t* ql, int nqe, const int32_t* qe,
                 const int32_t* order, const int32_t* par,
                 const int64_t* allow_off, const int32_t* allow_v, const uint8_t* allow_on,
                 int64_t max_emb, int32_t* emb_out, uint64_t* count_out, uint64_t* depth_out,
                 double* balg_out, int64_t node_budget, int nthreads, uint64_t limit) {
    if (k < 1 || k > OMAXK) return -1;
    int A[OMAXK][OMAXK];
    memset(A, 0, sizeof(A));
    for (int e = 0; e < nqe; e++) {
        int a = qe[2 * e], b = qe[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return -2;
        A[a][b] = A[b][a] = 1;
    }
    sctx c;
    memset(&c, 0, sizeof(c));
    c.g = g; c.k = k; c.ql = ql;
    if (order) {
        for (int i = 0; i < k; i++) c.order[i] = order[i];
    } else {
        int seen[OMAXK] = {0}, qh = 0, qt = 0;
        c.order[qt++] = 0; seen[0] = 1;
        while (qh < qt) {
            int u = c.order[qh++];
            for (int w = 0; w < k; w++)
                if (A[u][w] && !seen[w]) { seen[w] = 1; c.order[qt++] = w; }
        }
        if (qt != k) return -3;   /* disconnected query */
    }
    int pos[OMAXK];
    for (int i = 0; i < k; i++) pos[i] = -1;
    for (int i = 0; i < k; i++) {
        if (c.order[i] < 0 || c.order[i] >= k || pos[c.order[i]] >= 0) return -4;
        pos[c.order[i]] = i;
    }
    for (int d = 1; d < k; d++) {
        int u = c.order[d];
        int p = par ? par[d] : -1;
        if (p < 0) {
            for (int j = 0; j < d; j++) if (A[u][c.order[j]]) { p = j; break; }
        }
        if (p < 0 || p >= d || !A[u][c.order[p]]) return -3;
        c.par[d] = p;
        c.nb[d] = 0;
        for (int j = 0; j < d; j++)
            if (j != p && A[u][c.order[j]]) c.bn[d][c.nb[d]++] = j;
    }
    c.aoff = allow_off; c.av = allow_v; c.aon = allow_on;
    c.max_emb = max_emb; c.emb = emb_out;
    int64_t slot = 0;
    c.emb_slot = &slot;
    c.budget = node_budget;
    uint64_t found = 0;
    c.limit = limit;
    c.found = &found;

    /* root candidates: every vertex carrying the root's label */
    int ur = c.order[0];
    int64_t nr = 0;
    int32_t* roots = (int32_t*)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < g->n; v++)
        if (g->lab[v] == ql[ur] && allowed(&c, ur, (int32_t)v)) roots[nr++] = (int32_t)v;

    int want_balg = balg_out != NULL;
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    sacc* acc = (sacc*)calloc((size_t)nt, sizeof(sacc));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int32_t M[OMAXK];
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < nr; r++) {
            if (acc[t].over) continue;
            M[0] = roots[r];
            extend(&c, &acc[t], M, 1, want_balg);
        }
    }
    uint64_t cnt = 0;
    double balg[2] = {0.0, 0.0};
    int over = 0, limited = 0;
    if (depth_out) memset(depth_out, 0, (size_t)k * sizeof(uint64_t));
    for (int t = 0; t < nt; t++) {
        cnt += acc[t].count;
        balg[0] += acc[t].balg[0];
        balg[1] += acc[t].balg[1];
        over |= acc[t].over == 1;
        limited |= acc[t].over == 2;
        if (depth_out) for (int d = 0; d < k; d++) depth_out[d] += acc[t].depth[d];
    }
    *count_out = cnt;
    if (balg_out) { balg_out[0] = balg[0]; balg_out[1] = balg[1]; }
    free(acc); free(roots);
    if (over && !limited) return 1;
    return 0;
}

/*
 * Check rows of a candidate embedding list against Definition 1 directly:
 * labels, injectivity and every query edge present in G.  emb[rows][k] is
 * indexed by query vertex.  Returns the number of rows that fail.
 */
int64_t oracle_check_embeddings(const og* g, int k, const int32_t* ql, int nqe, const int32_t* qe,
                                int64_t rows, const int32_t* emb) {
    int64_t bad = 0;
    for (int64_t r = 0; r < rows; r++) {
        const int32_t* M = emb + r * k;
        int ok = 1;
        for (int u = 0; u < k && ok; u++) {
            if (M[u] < 0 || M[u] >= g->n || g->lab[M[u]] != ql[u]) ok = 0;
            for (int w = 0; w < u && ok; w++) if (M[w] == M[u]) ok = 0;
        }
        for (int e = 0; e < nqe && ok; e++)
            if (!has_edge(g, M[qe[2 * e]], M[qe[2 * e + 1]])) ok = 0;
        bad += !ok;
    }
    return bad;
}
