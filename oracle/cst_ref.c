/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain CPU restatement of the candidate search tree (CST) of Sec. IV-A
 * (Algorithm 1), of the query preparation it needs (root, BFS tree t_q,
 * path-based matching order) and of the workload estimate of Sec. IV-C.
 * It follows the paper's steps in its order, one loop per step, with the
 * readings below; it shares no code with the CUDA library.
 *
 * Readings of points the paper leaves open (each gives the same embeddings):
 *   filter   rule 0: C0(u) = { v : l_G(v) = l_q(u), d_G(v) >= d_q(u) }
 *            ("local features", Sec. IV-A: labels and degrees).
 *            rule 1 (neighbour label frequency, a stronger local feature):
 *            also, for every label l, v has at least as many neighbours
 *            labelled l as u has.  Sound: an embedding maps u's neighbours
 *            labelled l injectively onto neighbours of v labelled l.
 *   root     argmin over u of |C0(u)| / d_q(u), ties to the smaller id
 *            (k = 1: vertex 0).
 *   t_q      breadth-first from the root, neighbours in increasing id.
 *   top-down for u != root in BFS order: C(u) = { v in C0(u) : v adjacent to
 *            some v_p in C(u_p) } and N^{u_p}_u(v_p) = N_G(v_p) n C(u).
 *   bottom-up for u in reverse BFS order: each child list N^u_{u_c}(v) is cut
 *            to the (already refined) C(u_c); v stays in C(u) iff every such
 *            list is non-empty and (u is the root or v lies in some list of
 *            the parent).  refine rule 0: one pass, as written.
 *            refine rule 1 (the fixpoint refinement the paper leaves out,
 *            as CS-style filters do): v must also have, for every query
 *            neighbour w of u joined by a non-tree edge, a neighbour in C(w);
 *            the pass repeats until it removes nothing.  Sound: an
 *            embedding's image of u passes every test, so no embedding is
 *            lost; for a tree query with pairwise distinct labels the result
 *            is exactly the projections of the embedding set.
 *            refine rule 2: the same non-tree test in the single pass,
 *            against each set as it stands when u is reached (refined for
 *            vertices later in the BFS order, top-down for earlier ones);
 *            no repeat.  Between rule 1 and rule 0 as sets.
 *   order    rule 0 (the paper's path-based order, Sec. IV-B): depth-first
 *            preorder of t_q from the root, children visited in increasing
 *            (|C(u_c)|, u_c): whole root-to-leaf paths in turn.
 *            rule 1 (greedy; the paper's method takes any connected order,
 *            Sec. IV-B): after the root, repeatedly the unplaced vertex whose
 *            t_q parent is placed with the most query edges to placed
 *            vertices; ties to the smaller |C(u)|, then the smaller id.
 *            rule 2 (breadth-first): the BFS order of t_q itself, the order
 *            in which the tree was built.
 *            rule 3 (smallest candidate set first): after the root,
 *            repeatedly the unplaced vertex whose t_q parent is placed with
 *            the fewest candidates; ties to the smaller id.
 *            Every rule places every vertex after its t_q parent.
 *   non-tree for each query edge outside t_q, from its earlier endpoint u_j
 *            to its later endpoint u_i in the order: N^{u_j}_{u_i}(v) =
 *            N_G(v) n C(u_i) for v in C(u_j).  Only this direction is read
 *            when matching in that order.
 *   workload c_u(v) = 1 at leaves; c_u(v) = prod over children u' of the sum
 *            of c_{u'}(v') over v' in N^u_{u'}(v); W = sum over the root's
 *            candidates.  The product runs over the children of u in t_q.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    int64_t* off;
    int32_t* adj;
    int32_t* lab;
} og;   /* same layout as oracle.c */

#define CMAXK 64

typedef struct { int32_t* v; int64_t n, cap; } ivec;

static void iv_push(ivec* a, int32_t x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 8;
        a->v = (int32_t*)realloc(a->v, (size_t)a->cap * sizeof(int32_t));
    }
    a->v[a->n++] = x;
}

typedef struct {
    int k;
    int root;
    int parent[CMAXK];          /* query vertex -> parent in t_q (-1 root) */
    int bfs[CMAXK];             /* BFS order of t_q */
    int order[CMAXK];           /* matching order: position -> query vertex */
    int64_t c0n[CMAXK];         /* |C0(u)| */
    ivec cand[CMAXK];           /* C(u), sorted */
    ivec* tree[CMAXK];          /* tree[u][i] = N^{p(u)}_u(C(p(u))[i]) */
    int64_t tree_n[CMAXK];      /* rows in tree[u] (= |C(p(u))|) */
    int nnt;
    int nt_from[CMAXK * CMAXK / 2], nt_to[CMAXK * CMAXK / 2];
    ivec* nt[CMAXK * CMAXK / 2];  /* nt[e][i] = N^{from}_{to}(C(from)[i]) */
    int64_t nt_n[CMAXK * CMAXK / 2];
} ocst;

static int64_t find_sorted(const int32_t* a, int64_t n, int32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < n && a[lo] == x) ? lo : -1;
}

void oracle_cst_free(ocst* c) {
    if (!c) return;
    for (int u = 0; u < c->k; u++) {
        free(c->cand[u].v);
        if (c->tree[u]) {
            for (int64_t i = 0; i < c->tree_n[u]; i++) free(c->tree[u][i].v);
            free(c->tree[u]);
        }
    }
    for (int e = 0; e < c->nnt; e++) {
        for (int64_t i = 0; i < c->nt_n[e]; i++) free(c->nt[e][i].v);
        free(c->nt[e]);
    }
    free(c);
}

/*
 * Build the CST of q over G (Algorithm 1 with the readings above).
 * Returns a handle, or NULL on invalid or disconnected input.
 */
ocst* oracle_cst_build(const og* g, int k, const int32_t* ql, int nqe, const int32_t* qe, int order_rule,
                       int filter_rule, int refine_rule) {
    if (k < 1 || k > CMAXK || order_rule < 0 || order_rule > 3 || filter_rule < 0 || filter_rule > 1 ||
        refine_rule < 0 || refine_rule > 2)
        return NULL;
    int A[CMAXK][CMAXK];
    memset(A, 0, sizeof(A));
    int dq[CMAXK] = {0};
    for (int e = 0; e < nqe; e++) {
        int a = qe[2 * e], b = qe[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return NULL;
        if (!A[a][b]) { A[a][b] = A[b][a] = 1; dq[a]++; dq[b]++; }
    }
    ocst* c = (ocst*)calloc(1, sizeof(ocst));
    c->k = k;

    /* local-feature filter C0(u) */
    ivec c0[CMAXK];
    memset(c0, 0, sizeof(c0));
    for (int u = 0; u < k; u++) {
        /* rule 1: the labels of u's query neighbours and how often each occurs */
        int32_t nl[CMAXK];
        int need[CMAXK], nn = 0;
        for (int w = 0; w < k; w++) {
            if (!A[u][w]) continue;
            int t = 0;
            while (t < nn && nl[t] != ql[w]) t++;
            if (t == nn) { nl[nn] = ql[w]; need[nn] = 0; nn++; }
            need[t]++;
        }
        for (int64_t v = 0; v < g->n; v++) {
            if (g->lab[v] != ql[u] || g->off[v + 1] - g->off[v] < dq[u]) continue;
            if (filter_rule == 1) {
                int have[CMAXK] = {0}, ok = 1;
                for (int64_t i = g->off[v]; i < g->off[v + 1]; i++)
                    for (int t = 0; t < nn; t++)
                        if (g->lab[g->adj[i]] == nl[t]) have[t]++;
                for (int t = 0; t < nn; t++)
                    if (have[t] < need[t]) ok = 0;
                if (!ok) continue;
            }
            iv_push(&c0[u], (int32_t)v);
        }
        c->c0n[u] = c0[u].n;
    }

    /* root */
    int r = 0;
    if (k > 1) {
        for (int u = 1; u < k; u++)
            if (c0[u].n * (int64_t)dq[r] < c0[r].n * (int64_t)dq[u]) r = u;
    }
    c->root = r;

    /* BFS tree */
    int seen[CMAXK] = {0};
    int qh = 0, qt = 0;
    c->bfs[qt++] = r; seen[r] = 1; c->parent[r] = -1;
    while (qh < qt) {
        int u = c->bfs[qh++];
        for (int w = 0; w < k; w++)
            if (A[u][w] && !seen[w]) { seen[w] = 1; c->parent[w] = u; c->bfs[qt++] = w; }
    }
    if (qt != k) { for (int u = 0; u < k; u++) free(c0[u].v); free(c); return NULL; }

    /* top-down construction */
    uint8_t* mark = (uint8_t*)calloc((size_t)g->n + 1, 1);
    c->cand[r] = c0[r];
    c0[r].v = NULL;
    for (int t = 1; t < k; t++) {
        int u = c->bfs[t], p = c->parent[u];
        for (int64_t i = 0; i < c0[u].n; i++) mark[c0[u].v[i]] = 1;    /* member of C0(u) */
        c->tree_n[u] = c->cand[p].n;
        c->tree[u] = (ivec*)calloc((size_t)(c->cand[p].n > 0 ? c->cand[p].n : 1), sizeof(ivec));
        for (int64_t i = 0; i < c->cand[p].n; i++) {
            int32_t vp = c->cand[p].v[i];
            for (int64_t j = g->off[vp]; j < g->off[vp + 1]; j++) {
                int32_t v = g->adj[j];
                if (mark[v]) { iv_push(&c->tree[u][i], v); mark[v] = 2; }   /* 2: reached */
            }
        }
        for (int64_t i = 0; i < c0[u].n; i++) {
            int32_t v = c0[u].v[i];
            if (mark[v] == 2) iv_push(&c->cand[u], v);
            mark[v] = 0;
        }
        free(c0[u].v); c0[u].v = NULL;
    }
    free(mark);

    /* bottom-up refinement (rule 1: repeated, with the non-tree test, until
     * a pass removes nothing) */
    int64_t removed;
    do {
    removed = 0;
    for (int t = k - 1; t >= 0; t--) {
        int u = c->bfs[t];
        int64_t nu = c->cand[u].n;
        uint8_t* keep = (uint8_t*)malloc((size_t)(nu > 0 ? nu : 1));
        /* haspar[i]: C(u)[i] lies in some list N^{u_p}_u(v_p), v_p in C(u_p) */
        uint8_t* haspar = (uint8_t*)calloc((size_t)(nu > 0 ? nu : 1), 1);
        if (u != r)
            for (int64_t a = 0; a < c->tree_n[u]; a++)
                for (int64_t j = 0; j < c->tree[u][a].n; j++) {
                    int64_t x = find_sorted(c->cand[u].v, nu, c->tree[u][a].v[j]);
                    if (x >= 0) haspar[x] = 1;
                }
        for (int64_t i = 0; i < nu; i++) {
            int32_t v = c->cand[u].v[i];
            int ok = 1;
            for (int w = 0; w < k; w++) {
                if (c->parent[w] != u) continue;
                ivec* L = &c->tree[w][i];
                int64_t o = 0;
                for (int64_t j = 0; j < L->n; j++)
                    if (find_sorted(c->cand[w].v, c->cand[w].n, L->v[j]) >= 0) L->v[o++] = L->v[j];
                L->n = o;
                if (o == 0) ok = 0;
            }
            if (ok && u != r && !haspar[i]) ok = 0;
            if (ok && refine_rule >= 1)
                for (int w = 0; w < k && ok; w++) {
                    if (!A[u][w] || c->parent[w] == u || c->parent[u] == w) continue;   /* tree edge */
                    int any = 0;
                    for (int64_t j = g->off[v]; j < g->off[v + 1] && !any; j++)
                        if (find_sorted(c->cand[w].v, c->cand[w].n, g->adj[j]) >= 0) any = 1;
                    if (!any) ok = 0;
                }
            keep[i] = (uint8_t)ok;
            if (!ok) removed++;
        }
        /* drop invalid candidates together with their lists */
        int64_t o = 0;
        for (int64_t i = 0; i < nu; i++) {
            if (keep[i]) {
                c->cand[u].v[o] = c->cand[u].v[i];
                for (int w = 0; w < k; w++)
                    if (c->parent[w] == u) {
                        if (o != i) { c->tree[w][o] = c->tree[w][i]; c->tree[w][i].v = NULL; c->tree[w][i].n = 0; c->tree[w][i].cap = 0; }
                    }
                o++;
            } else {
                for (int w = 0; w < k; w++)
                    if (c->parent[w] == u) { free(c->tree[w][i].v); c->tree[w][i].v = NULL; c->tree[w][i].n = 0; c->tree[w][i].cap = 0; }
            }
        }
        c->cand[u].n = o;
        for (int w = 0; w < k; w++) if (c->parent[w] == u) c->tree_n[w] = o;
        free(keep); free(haspar);
    }
    } while (refine_rule == 1 && removed > 0);

    /* matching order, rule 2: the BFS order of t_q */
    if (order_rule == 2) {
        for (int i = 0; i < k; i++) c->order[i] = c->bfs[i];
    } else
    /* matching order, rule 3: the placeable vertex with the fewest candidates */
    if (order_rule == 3) {
        int placed[CMAXK] = {0};
        c->order[0] = r;
        placed[r] = 1;
        for (int no = 1; no < k; no++) {
            int best = -1;
            for (int u = 0; u < k; u++) {
                if (placed[u] || !placed[c->parent[u]]) continue;
                if (best < 0 || c->cand[u].n < c->cand[best].n || (c->cand[u].n == c->cand[best].n && u < best)) best = u;
            }
            c->order[no] = best;
            placed[best] = 1;
        }
    } else
    /* matching order, rule 1: greedy by edges to the placed vertices */
    if (order_rule == 1) {
        int placed[CMAXK] = {0};
        c->order[0] = r;
        placed[r] = 1;
        for (int no = 1; no < k; no++) {
            int best = -1, bb = -1;
            for (int u = 0; u < k; u++) {
                if (placed[u] || !placed[c->parent[u]]) continue;
                int b = 0;
                for (int w = 0; w < k; w++) if (placed[w] && A[u][w]) b++;
                if (best < 0 || b > bb ||
                    (b == bb && (c->cand[u].n < c->cand[best].n || (c->cand[u].n == c->cand[best].n && u < best)))) {
                    best = u;
                    bb = b;
                }
            }
            c->order[no] = best;
            placed[best] = 1;
        }
    } else
    /* matching order, rule 0: DFS preorder, children by (|C|, id) */
    {
        int stack[CMAXK], sp = 0, no = 0;
        stack[sp++] = r;
        while (sp) {
            int u = stack[--sp];
            c->order[no++] = u;
            int ch[CMAXK], nc = 0;
            for (int w = 0; w < k; w++) if (c->parent[w] == u) ch[nc++] = w;
            for (int a = 1; a < nc; a++)      /* insertion sort by (|C|, id) */
                for (int b = a; b > 0; b--) {
                    int x = ch[b - 1], y = ch[b];
                    if (c->cand[y].n < c->cand[x].n || (c->cand[y].n == c->cand[x].n && y < x)) { ch[b - 1] = y; ch[b] = x; }
                    else break;
                }
            for (int a = nc - 1; a >= 0; a--) stack[sp++] = ch[a];   /* smallest popped first */
        }
    }

    /* non-tree candidate edges, earlier -> later endpoint in the order */
    int pos[CMAXK];
    for (int i = 0; i < k; i++) pos[c->order[i]] = i;
    for (int i = 0; i < k; i++) {
        int ui = c->order[i];
        for (int j = 0; j < i; j++) {
            int uj = c->order[j];
            if (!A[ui][uj] || c->parent[ui] == uj || c->parent[uj] == ui) continue;
            int e = c->nnt++;
            c->nt_from[e] = uj; c->nt_to[e] = ui;
            c->nt_n[e] = c->cand[uj].n;
            c->nt[e] = (ivec*)calloc((size_t)(c->cand[uj].n > 0 ? c->cand[uj].n : 1), sizeof(ivec));
            for (int64_t a = 0; a < c->cand[uj].n; a++) {
                int32_t v = c->cand[uj].v[a];
                for (int64_t b = g->off[v]; b < g->off[v + 1]; b++)
                    if (find_sorted(c->cand[ui].v, c->cand[ui].n, g->adj[b]) >= 0) iv_push(&c->nt[e][a], g->adj[b]);
            }
        }
    }
    (void)pos;
    return c;
}

/* ---- accessors (arrays are copied into caller buffers) ---- */

int oracle_cst_root(const ocst* c) { return c->root; }
void oracle_cst_tree_shape(const ocst* c, int32_t* parent, int32_t* bfs, int32_t* order) {
    for (int u = 0; u < c->k; u++) { parent[u] = c->parent[u]; bfs[u] = c->bfs[u]; order[u] = c->order[u]; }
}
int64_t oracle_cst_c0_count(const ocst* c, int u) { return c->c0n[u]; }
int64_t oracle_cst_cand_count(const ocst* c, int u) { return c->cand[u].n; }
void oracle_cst_cand(const ocst* c, int u, int32_t* out) {
    memcpy(out, c->cand[u].v, (size_t)c->cand[u].n * sizeof(int32_t));
}
/* tree lists into u: rows = |C(parent(u))|; total entries returned */
int64_t oracle_cst_tree_total(const ocst* c, int u) {
    int64_t s = 0;
    for (int64_t i = 0; i < c->tree_n[u]; i++) s += c->tree[u][i].n;
    return s;
}
void oracle_cst_tree(const ocst* c, int u, int64_t* off, int32_t* vals) {
    off[0] = 0;
    for (int64_t i = 0; i < c->tree_n[u]; i++) {
        memcpy(vals + off[i], c->tree[u][i].v, (size_t)c->tree[u][i].n * sizeof(int32_t));
        off[i + 1] = off[i] + c->tree[u][i].n;
    }
}
int oracle_cst_nt_count(const ocst* c) { return c->nnt; }
void oracle_cst_nt_edge(const ocst* c, int e, int32_t* from, int32_t* to) { *from = c->nt_from[e]; *to = c->nt_to[e]; }
int64_t oracle_cst_nt_total(const ocst* c, int e) {
    int64_t s = 0;
    for (int64_t i = 0; i < c->nt_n[e]; i++) s += c->nt[e][i].n;
    return s;
}
void oracle_cst_nt(const ocst* c, int e, int64_t* off, int32_t* vals) {
    off[0] = 0;
    for (int64_t i = 0; i < c->nt_n[e]; i++) {
        memcpy(vals + off[i], c->nt[e][i].v, (size_t)c->nt[e][i].n * sizeof(int32_t));
        off[i + 1] = off[i] + c->nt[e][i].n;
    }
}

/* ---- workload estimate (Sec. IV-C) ---- */

static uint64_t sat_add(uint64_t a, uint64_t b) { return (a > UINT64_MAX - b) ? UINT64_MAX : a + b; }
static uint64_t sat_mul(uint64_t a, uint64_t b) {
    if (a == 0 || b == 0) return 0;
    return (a > UINT64_MAX / b) ? UINT64_MAX : a * b;
}

/*
 * c_u(v) for every candidate, in both float64 and saturating uint64, then
 * W = sum over the root's candidates.  cu_f / cu_i (nullable) receive c for
 * query vertex `dump_u` (|C(dump_u)| entries).
 */
void oracle_cst_workload(const ocst* c, double* w_f, uint64_t* w_i, int dump_u, double* cu_f, uint64_t* cu_i) {
    int k = c->k;
    double* cf[CMAXK];
    uint64_t* ci[CMAXK];
    for (int t = k - 1; t >= 0; t--) {
        int u = c->bfs[t];
        int64_t nu = c->cand[u].n;
        cf[u] = (double*)malloc((size_t)(nu > 0 ? nu : 1) * sizeof(double));
        ci[u] = (uint64_t*)malloc((size_t)(nu > 0 ? nu : 1) * sizeof(uint64_t));
        for (int64_t i = 0; i < nu; i++) { cf[u][i] = 1.0; ci[u][i] = 1; }
        for (int w = 0; w < k; w++) {
            if (c->parent[w] != u) continue;
            for (int64_t i = 0; i < nu; i++) {
                double sf = 0.0;
                uint64_t si = 0;
                const ivec* L = &c->tree[w][i];
                for (int64_t j = 0; j < L->n; j++) {
                    int64_t x = find_sorted(c->cand[w].v, c->cand[w].n, L->v[j]);
                    sf += cf[w][x];
                    si = sat_add(si, ci[w][x]);
                }
                cf[u][i] *= sf;
                ci[u][i] = sat_mul(ci[u][i], si);
            }
        }
    }
    double Wf = 0.0;
    uint64_t Wi = 0;
    for (int64_t i = 0; i < c->cand[c->root].n; i++) { Wf += cf[c->root][i]; Wi = sat_add(Wi, ci[c->root][i]); }
    *w_f = Wf; *w_i = Wi;
    if (dump_u >= 0 && dump_u < k) {
        if (cu_f) memcpy(cu_f, cf[dump_u], (size_t)c->cand[dump_u].n * sizeof(double));
        if (cu_i) memcpy(cu_i, ci[dump_u], (size_t)c->cand[dump_u].n * sizeof(uint64_t));
    }
    for (int u = 0; u < k; u++) { free(cf[u]); free(ci[u]); }
}

/* ---- partition (Algorithm 2, Sec. IV-B) ----
 *
 * Readings:
 *   size     The partition factor is driven by the workload estimate:
 *            k = min(ceil(W'/delta_w), |C'(u)|), with W' the estimate of
 *            Sec. IV-C evaluated on the partitioned tree CST' in saturating
 *            uint64 arithmetic (exact below 2^64).  The paper's delta_S and
 *            delta_D bound BRAM bytes and FPGA read ports; W' bounds the work
 *            one chunk holds.
 *   split    C'(u) is cut into k contiguous runs of its id-sorted list,
 *            run i = [floor(i n/k), floor((i+1) n/k)).
 *   restrict positions before u keep their sets; u keeps the run; every
 *            later position keeps the candidates listed by some kept
 *            candidate of its t_q parent (processed in matching order).
 *   recurse  a run with W' <= delta_w is a chunk (W' = 0 runs hold no
 *            embedding and are dropped); otherwise a run of one candidate
 *            moves on to the next position, and a longer run is split again.
 *   fixed    when a run of one candidate v at position j moves on, v joins
 *            the fixed prefix; if v equals the candidate fixed at an earlier
 *            position, or lacks a CST edge to the candidate fixed at an
 *            earlier non-tree neighbour, the part holds no embedding and is
 *            dropped (the CST validity rule applied to single candidates).
 *   cap      runs are processed level by level (all runs of one depth of the
 *            recursion, in order); a level whose chunks plus new parts
 *            would pass max_chunks caps each split at
 *            max(1, (max_chunks - chunks so far - runs finishing) /
 *            runs splitting) parts, and those parts become the last chunks
 *            as they are (W' may exceed delta_w; W' = 0 parts included),
 *            which keeps them disjoint and complete.
 *   sample   optional: a run produced by a split into k parts is kept iff
 *            u01(id) < min(1, c/k), c = c_root at the first position and
 *            c_deep later (c <= 0 keeps every run).  id(root) = mix64(seed),
 *            id(run i) = mix64(id(parent) + (i+1) * 0x9E3779B97F4A7C15), with
 *            mix64 the splitmix64 finaliser and u01(x) = (x >> 11) * 2^-53.
 * Since every position before u is a single candidate when u is split, a
 * chunk is (j, the candidates of positions 0..j-1, a run [a, b) of the list
 * L_j), where L_j is C(root) for j = 0 and otherwise the tree list of the
 * candidate at the parent position of position j.
 */

static uint64_t pmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    int j;
    int32_t prefix[CMAXK];      /* global ids of positions 0..j-1 */
    int64_t a, b;
    uint64_t w;
    uint64_t id;
} ochunk;

typedef struct {
    const ocst* c;
    int pos[CMAXK];             /* query vertex -> position */
    uint64_t delta_w;
    double c_root, c_deep;
    ochunk* out;
    int64_t nout, cap;
    int64_t max_chunks;
    int overflow;
} pctx;

/* the list L_j of a chunk: pointer + length (global ids, sorted) */
static const int32_t* chunk_list(const pctx* P, int j, const int32_t* prefix, int64_t* len) {
    const ocst* c = P->c;
    int u = c->order[j];
    if (j == 0) { *len = c->cand[u].n; return c->cand[u].v; }
    int p = c->parent[u];
    int64_t row = find_sorted(c->cand[p].v, c->cand[p].n, prefix[P->pos[p]]);
    if (row < 0) { *len = 0; return NULL; }
    *len = c->tree[u][row].n;
    return c->tree[u][row].v;
}

/* W' of the partitioned tree: restricted candidate sets, then the DP of
 * Sec. IV-C over them, in saturating uint64. */
static uint64_t restricted_w(const pctx* P, int j, const int32_t* prefix, const int32_t* run, int64_t nrun) {
    const ocst* c = P->c;
    int k = c->k;
    uint8_t* on[CMAXK];
    for (int u = 0; u < k; u++) on[u] = (uint8_t*)calloc((size_t)(c->cand[u].n > 0 ? c->cand[u].n : 1), 1);
    for (int i = 0; i < k; i++) {
        int u = c->order[i];
        if (i < j) {
            int64_t x = find_sorted(c->cand[u].v, c->cand[u].n, prefix[i]);
            if (x >= 0) on[u][x] = 1;
        } else if (i == j) {
            for (int64_t r = 0; r < nrun; r++) {
                int64_t x = find_sorted(c->cand[u].v, c->cand[u].n, run[r]);
                if (x >= 0) on[u][x] = 1;
            }
        } else {
            int p = c->parent[u];
            for (int64_t a = 0; a < c->cand[p].n; a++) {
                if (!on[p][a]) continue;
                for (int64_t t = 0; t < c->tree[u][a].n; t++) {
                    int64_t x = find_sorted(c->cand[u].v, c->cand[u].n, c->tree[u][a].v[t]);
                    if (x >= 0) on[u][x] = 1;
                }
            }
        }
    }
    uint64_t* cv[CMAXK];
    for (int t = k - 1; t >= 0; t--) {
        int u = c->bfs[t];
        int64_t nu = c->cand[u].n;
        cv[u] = (uint64_t*)malloc((size_t)(nu > 0 ? nu : 1) * sizeof(uint64_t));
        for (int64_t i = 0; i < nu; i++) cv[u][i] = on[u][i] ? 1 : 0;
        for (int w = 0; w < k; w++) {
            if (c->parent[w] != u) continue;
            for (int64_t i = 0; i < nu; i++) {
                if (!on[u][i]) continue;
                uint64_t s = 0;
                const ivec* L = &c->tree[w][i];
                for (int64_t t = 0; t < L->n; t++) {
                    int64_t x = find_sorted(c->cand[w].v, c->cand[w].n, L->v[t]);
                    if (x >= 0 && on[w][x]) s = sat_add(s, cv[w][x]);
                }
                cv[u][i] = sat_mul(cv[u][i], s);
            }
        }
    }
    uint64_t W = 0;
    int r = c->root;
    for (int64_t i = 0; i < c->cand[r].n; i++) if (on[r][i]) W = sat_add(W, cv[r][i]);
    for (int u = 0; u < k; u++) { free(on[u]); free(cv[u]); }
    return W;
}

/* may candidate v sit at position j after the fixed prefix[0..j-1]? */
static int prefix_ok(const pctx* P, int j, const int32_t* prefix, int32_t v) {
    const ocst* c = P->c;
    int u = c->order[j];
    for (int p = 0; p < j; p++)
        if (prefix[p] == v) return 0;
    for (int e = 0; e < c->nnt; e++) {
        if (c->nt_to[e] != u) continue;
        int f = c->nt_from[e];
        int64_t row = find_sorted(c->cand[f].v, c->cand[f].n, prefix[P->pos[f]]);
        if (row < 0 || find_sorted(c->nt[e][row].v, c->nt[e][row].n, v) < 0) return 0;
    }
    return 1;
}

static void p_emit(pctx* P, const ochunk* ch) {
    if (P->nout == P->cap) {
        P->cap = P->cap ? 2 * P->cap : 64;
        P->out = (ochunk*)realloc(P->out, (size_t)P->cap * sizeof(ochunk));
    }
    P->out[P->nout++] = *ch;
}

/* Move runs of one candidate on to the next position (same W'), checking
 * the newly fixed candidate.  Returns 0 drop, 1 chunk, 2 split (kk parts). */
static int p_classify(const pctx* P, ochunk* ch, uint64_t* kk_out) {
    const ocst* c = P->c;
    for (;;) {
        if (ch->w == 0) return 0;
        if (ch->w <= P->delta_w) return 1;
        int64_t n = ch->b - ch->a;
        int64_t len;
        const int32_t* L = chunk_list(P, ch->j, ch->prefix, &len);
        if (n == 1) {
            if (ch->j + 1 >= c->k) return 1;                 /* cannot split further */
            if (!prefix_ok(P, ch->j, ch->prefix, L[ch->a])) return 0;
            ch->prefix[ch->j] = L[ch->a];
            ch->j += 1;
            chunk_list(P, ch->j, ch->prefix, &len);
            ch->a = 0; ch->b = len;
            continue;                                       /* same tree, next position */
        }
        uint64_t kk = ch->w / P->delta_w + (ch->w % P->delta_w != 0);
        if (kk > (uint64_t)n) kk = (uint64_t)n;
        *kk_out = kk;
        return 2;
    }
}

static int p_keep(const pctx* P, int j, uint64_t kk, uint64_t id) {
    double cs = j == 0 ? P->c_root : P->c_deep;
    double tau = cs <= 0.0 ? 2.0 : (cs / (double)kk < 1.0 ? cs / (double)kk : 2.0);
    return !(tau <= 1.0 && (double)(id >> 11) * (1.0 / 9007199254740992.0) >= tau);
}

/* Level by level: every pending run is moved on / classified; a level whose
 * chunks and parts would pass max_chunks instead turns its live runs into
 * chunks as they are. */
static void p_levels(pctx* P, ochunk root) {
    ochunk* cur = (ochunk*)malloc(sizeof(ochunk));
    int64_t ncur = 1;
    cur[0] = root;
    while (ncur > 0 && !P->overflow) {
        int* act = (int*)malloc((size_t)ncur * sizeof(int));
        uint64_t* kk = (uint64_t*)calloc((size_t)ncur, sizeof(uint64_t));
        int64_t ne = 0, np = 0, nl = 0;
        for (int64_t t = 0; t < ncur; t++) {
            act[t] = p_classify(P, &cur[t], &kk[t]);
            ne += act[t] == 1;
            nl += act[t] != 0;
            if (act[t] == 2)
                for (uint64_t i = 0; i < kk[t]; i++)
                    np += p_keep(P, cur[t].j, kk[t], pmix(cur[t].id + (i + 1) * 0x9E3779B97F4A7C15ull));
        }
        int last = 0;
        if (P->nout + ne + np > P->max_chunks) {
            /* cap every split at an even share of the room left; its parts
             * are the last chunks */
            int64_t nsplit = nl - ne, room = P->max_chunks - P->nout - ne;
            uint64_t kcap = (uint64_t)((nsplit > 0 && room / nsplit > 1) ? room / nsplit : 1);
            np = 0;
            for (int64_t t = 0; t < ncur; t++) {
                if (act[t] != 2) continue;
                if (kk[t] > kcap) kk[t] = kcap;
                for (uint64_t i = 0; i < kk[t]; i++)
                    np += p_keep(P, cur[t].j, kk[t], pmix(cur[t].id + (i + 1) * 0x9E3779B97F4A7C15ull));
            }
            last = 1;
        }
        ochunk* nxt = (ochunk*)malloc((size_t)(np > 0 ? np : 1) * sizeof(ochunk));
        int64_t o = 0;
        for (int64_t t = 0; t < ncur; t++) {
            if (act[t] == 1) p_emit(P, &cur[t]);
            if (act[t] != 2) continue;
            ochunk* ch = &cur[t];
            int64_t n = ch->b - ch->a, len;
            const int32_t* L = chunk_list(P, ch->j, ch->prefix, &len);
            for (uint64_t i = 0; i < kk[t]; i++) {
                uint64_t id = pmix(ch->id + (i + 1) * 0x9E3779B97F4A7C15ull);
                if (!p_keep(P, ch->j, kk[t], id)) continue;
                ochunk sub = *ch;
                sub.a = ch->a + (int64_t)((__uint128_t)i * (uint64_t)n / kk[t]);
                sub.b = ch->a + (int64_t)((__uint128_t)(i + 1) * (uint64_t)n / kk[t]);
                sub.id = id;
                sub.w = restricted_w(P, sub.j, sub.prefix, L + sub.a, sub.b - sub.a);
                nxt[o++] = sub;
            }
        }
        free(act); free(kk); free(cur);
        cur = nxt;
        ncur = o;
        if (last) {
            for (int64_t t = 0; t < ncur; t++) p_emit(P, &cur[t]);
            ncur = 0;
        }
    }
    free(cur);
}

/*
 * Partition the CST (Algorithm 2 with the readings above).  Chunks are
 * written level by level, in order within a level: j_out[i],
 * prefix_out[i][k] (global ids, entries >= j unused), a_out/b_out, w_out
 * (W'), id_out.  Output arrays need room for max_chunks entries.  Returns
 * the chunk count.
 */
int64_t oracle_cst_partition(const ocst* c, uint64_t delta_w, double c_root, double c_deep, uint64_t seed,
                             int64_t max_chunks, int32_t* j_out, int32_t* prefix_out, int64_t* a_out,
                             int64_t* b_out, uint64_t* w_out, uint64_t* id_out) {
    pctx P;
    memset(&P, 0, sizeof(P));
    P.c = c; P.delta_w = delta_w ? delta_w : 1; P.c_root = c_root; P.c_deep = c_deep; P.max_chunks = max_chunks;
    for (int i = 0; i < c->k; i++) P.pos[c->order[i]] = i;
    ochunk root;
    memset(&root, 0, sizeof(root));
    root.j = 0; root.a = 0; root.b = c->cand[c->root].n; root.id = pmix(seed);
    double wf; uint64_t wi;
    oracle_cst_workload(c, &wf, &wi, -1, NULL, NULL);
    root.w = wi;
    if (root.b > 0) p_levels(&P, root);
    for (int64_t i = 0; i < P.nout; i++) {
        j_out[i] = P.out[i].j;
        for (int t = 0; t < c->k; t++) prefix_out[i * c->k + t] = t < P.out[i].j ? P.out[i].prefix[t] : -1;
        a_out[i] = P.out[i].a; b_out[i] = P.out[i].b; w_out[i] = P.out[i].w; id_out[i] = P.out[i].id;
    }
    int64_t n = P.nout;
    free(P.out);
    return n;
}

/* W' of one chunk given as (j, prefix global ids, run global ids). */
uint64_t oracle_cst_chunk_w(const ocst* c, int j, const int32_t* prefix, const int32_t* run, int64_t nrun) {
    pctx P;
    memset(&P, 0, sizeof(P));
    P.c = c;
    for (int i = 0; i < c->k; i++) P.pos[c->order[i]] = i;
    return restricted_w(&P, j, prefix, run, nrun);
}
