/*
 * Seeded synthetic inputs for the subgraph-matching workloads: data graphs
 * (Erdos-Renyi, Chung-Lu power law, R-MAT), vertex labels (uniform, Zipf) and
 * connected query graphs extracted from a data graph by random walk.
 *
 * This file holds no part of the matching method itself: no candidate
 * filtering, no search, no counting.  It only draws numbers.  Both the CUDA
 * library and the CPU oracle are fed from here.
 *
 * Every random number is a pure function of (seed, stream, counter) through
 * the splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), so the output does not depend on thread
 * count or on the host architecture.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rkey(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed) ^ (stream * 0xD1B54A32D192ED03ull));
}

static inline uint64_t rnd(uint64_t key, uint64_t ctr) {
    return mix64(key + ctr * 0x9E3779B97F4A7C15ull);
}

static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static inline uint64_t below(uint64_t r, uint64_t n) {
    return (uint64_t)(((__uint128_t)r * (__uint128_t)n) >> 64);
}

/* ------------------------------------------------- stable radix sort */

/* Sorts key[0..n) ascending and carries val[] along, stable (equal keys
 * keep their input order).  LSD radix, 16-bit digits, passes only over the
 * bits that vary.  Each pass splits the arrays into one contiguous range per
 * thread; every thread counts its digits, the offsets are laid out digit by
 * digit and, within a digit, thread by thread, and every thread scatters its
 * range in order -- so the result does not depend on the number of
 * threads. */
static int sort_kv(uint64_t* key, uint32_t* val, int64_t n) {
    if (n <= 1) return 0;
    uint64_t kmax = 0;
#pragma omp parallel for reduction(| : kmax) schedule(static)
    for (int64_t i = 0; i < n; i++) kmax |= key[i];
    int bits = 0;
    while (bits < 64 && (kmax >> bits)) bits++;
    int T = omp_get_max_threads();
    if (T < 1) T = 1;
    if (T > 64) T = 64;
    if (n < (int64_t)T * 65536) T = 1;            /* small inputs: one range */
    uint64_t* tk = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    uint32_t* tv = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    int64_t* cnt = (int64_t*)malloc((size_t)T * 65536 * sizeof(int64_t));
    if (!tk || !tv || !cnt) { free(tk); free(tv); free(cnt); return -1; }
    uint64_t* xk = key; uint32_t* xv = val; uint64_t* yk = tk; uint32_t* yv = tv;
    for (int sh = 0; sh < bits; sh += 16) {
        int used = T;
#pragma omp parallel num_threads(T)
        {
            const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#pragma omp single
            used = nt;
            const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* c = cnt + (int64_t)t * 65536;
            memset(c, 0, 65536 * sizeof(int64_t));
            for (int64_t i = lo; i < hi; i++) c[(xk[i] >> sh) & 0xFFFF]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t s = 0;
                for (int d = 0; d < 65536; d++)
                    for (int u = 0; u < used; u++) {
                        int64_t x = cnt[(int64_t)u * 65536 + d];
                        cnt[(int64_t)u * 65536 + d] = s;
                        s += x;
                    }
            }
            for (int64_t i = lo; i < hi; i++) {
                int64_t o = c[(xk[i] >> sh) & 0xFFFF]++;
                yk[o] = xk[i];
                yv[o] = xv[i];
            }
        }
        uint64_t* t1 = xk; xk = yk; yk = t1;
        uint32_t* t2 = xv; xv = yv; yv = t2;
    }
    if (xk != key) {
        memcpy(key, xk, (size_t)n * sizeof(uint64_t));
        memcpy(val, xv, (size_t)n * sizeof(uint32_t));
    }
    free(tk); free(tv); free(cnt);
    return 0;
}

/* ------------------------------------------- unique-edge accumulation */

/*
 * Edge sampler callback: writes candidate edge number `ctr` (0-based) into
 * (*s, *d).  Candidates are drawn in counter order; the first m distinct
 * non-loop pairs (as unordered pairs) are kept, in first-occurrence order.
 */
typedef void (*edge_fn)(const void* ctx, uint64_t ctr, int32_t* s, int32_t* d);

static int unique_edges(edge_fn fn, const void* ctx, int64_t m, int32_t* out /*[m][2]*/) {
    int64_t cap = m + m / 8 + 1024;
    for (int attempt = 0; attempt < 40; attempt++) {
        if (cap >= (int64_t)0xFFFFFFFFll) return -2;
        int32_t* es = (int32_t*)malloc((size_t)cap * 2 * sizeof(int32_t));
        uint64_t* key = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
        uint32_t* idx = (uint32_t*)malloc((size_t)cap * sizeof(uint32_t));
        uint8_t* keep = (uint8_t*)calloc((size_t)cap, 1);
        if (!es || !key || !idx || !keep) { free(es); free(key); free(idx); free(keep); return -1; }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cap; i++) {
            int32_t s, d;
            fn(ctx, (uint64_t)i, &s, &d);
            es[2 * i] = s; es[2 * i + 1] = d;
            uint64_t lo = (uint64_t)(s < d ? s : d), hi = (uint64_t)(s < d ? d : s);
            key[i] = (s == d) ? UINT64_MAX : ((lo << 32) | hi);
            idx[i] = (uint32_t)i;
        }
        if (sort_kv(key, idx, cap) != 0) { free(es); free(key); free(idx); free(keep); return -1; }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < cap; i++) {               /* loops (UINT64_MAX) sort last */
            uint64_t k = key[i];
            if (k != UINT64_MAX && (i == 0 || key[i - 1] != k)) keep[idx[i]] = 1;   /* first occurrence */
        }
        int64_t got = 0;
        for (int64_t i = 0; i < cap && got < m; i++)
            if (keep[i]) { out[2 * got] = es[2 * i]; out[2 * got + 1] = es[2 * i + 1]; got++; }
        free(es); free(key); free(idx); free(keep);
        if (got == m) return 0;
        cap = cap + cap / 2 + (m - got) * 2;
    }
    return -3;
}

/* ------------------------------------------------------ Erdos-Renyi */

typedef struct { uint64_t key; int64_t n; } er_ctx;

static void er_edge(const void* c, uint64_t ctr, int32_t* s, int32_t* d) {
    const er_ctx* x = (const er_ctx*)c;
    *s = (int32_t)below(rnd(x->key, 2 * ctr), (uint64_t)x->n);
    *d = (int32_t)below(rnd(x->key, 2 * ctr + 1), (uint64_t)x->n);
}

/* m distinct uniform edges over n vertices (G(n, m) model). */
int synth_er_edges(int64_t n, int64_t m, uint64_t seed, int32_t* out) {
    if (n < 2 || m < 0 || m > n * (n - 1) / 2) return -4;
    er_ctx c = {rkey(seed, 1), n};
    return unique_edges(er_edge, &c, m, out);
}

/* ---------------------------------------------------------- Chung-Lu */

typedef struct { uint64_t key; int64_t n; const double* cdf; } cl_ctx;

static int32_t cdf_pick(const double* cdf, int64_t n, double x) {
    int64_t lo = 0, hi = n - 1;            /* first i with cdf[i] > x */
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > x) hi = mid; else lo = mid + 1;
    }
    return (int32_t)lo;
}

static void cl_edge(const void* c, uint64_t ctr, int32_t* s, int32_t* d) {
    const cl_ctx* x = (const cl_ctx*)c;
    *s = cdf_pick(x->cdf, x->n, u01(rnd(x->key, 2 * ctr)));
    *d = cdf_pick(x->cdf, x->n, u01(rnd(x->key, 2 * ctr + 1)));
}

/* Chung-Lu: both endpoints drawn with probability proportional to
 * w_i = (i+1)^(-1/(gamma-1)), giving a degree tail with exponent gamma. */
int synth_chung_lu_edges(int64_t n, int64_t m, double gamma, uint64_t seed, int32_t* out) {
    if (n < 2 || m < 0 || gamma <= 1.0) return -4;
    double* cdf = (double*)malloc((size_t)n * sizeof(double));
    if (!cdf) return -1;
    double e = -1.0 / (gamma - 1.0), acc = 0.0;
    for (int64_t i = 0; i < n; i++) { acc += pow((double)(i + 1), e); cdf[i] = acc; }
    for (int64_t i = 0; i < n; i++) cdf[i] /= acc;
    cdf[n - 1] = 2.0; /* guard: every x in [0,1) lands */
    cl_ctx c = {rkey(seed, 2), n, cdf};
    int rc = unique_edges(cl_edge, &c, m, out);
    free(cdf);
    return rc;
}

/* ------------------------------------------------------------- R-MAT */

typedef struct { uint64_t key; int scale; double a, ab, abc; const int32_t* perm; } rmat_ctx;

static void rmat_edge(const void* c, uint64_t ctr, int32_t* s, int32_t* d) {
    const rmat_ctx* x = (const rmat_ctx*)c;
    uint32_t src = 0, dst = 0;
    for (int lev = 0; lev < x->scale; lev++) {
        double r = u01(rnd(x->key, ctr * 64 + (uint64_t)lev));
        uint32_t bs, bd;
        if (r < x->a) { bs = 0; bd = 0; }
        else if (r < x->ab) { bs = 0; bd = 1; }
        else if (r < x->abc) { bs = 1; bd = 0; }
        else { bs = 1; bd = 1; }
        src = (src << 1) | bs; dst = (dst << 1) | bd;
    }
    *s = x->perm[src]; *d = x->perm[dst];
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with quadrant probabilities
 * a, b, c, d = 1-a-b-c; vertex ids are shuffled by a seeded permutation
 * (as in Graph500) so that degree is not tied to id. */
int synth_rmat_edges(int scale, int64_t m, double a, double b, double c, uint64_t seed, int32_t* out) {
    if (scale < 1 || scale > 30 || m < 0) return -4;
    int64_t n = (int64_t)1 << scale;
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return -1;
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    uint64_t pk = rkey(seed, 4);
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)below(rnd(pk, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    rmat_ctx x = {rkey(seed, 3), scale, a, a + b, a + b + c, perm};
    int rc = unique_edges(rmat_edge, &x, m, out);
    free(perm);
    return rc;
}

/* ------------------------------------------------------------ labels */

int synth_labels_uniform(int64_t n, int32_t L, uint64_t seed, int32_t* out) {
    if (L < 1) return -4;
    uint64_t k = rkey(seed, 5);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) out[i] = (int32_t)below(rnd(k, (uint64_t)i), (uint64_t)L);
    return 0;
}

/* Zipf(s) over L labels: P(label = i) proportional to 1/(i+1)^s, label 0 the
 * most frequent; drawn independently of the vertex's degree. */
int synth_labels_zipf(int64_t n, int32_t L, double s, uint64_t seed, int32_t* out) {
    if (L < 1) return -4;
    double* cdf = (double*)malloc((size_t)L * sizeof(double));
    if (!cdf) return -1;
    double acc = 0.0;
    for (int i = 0; i < L; i++) { acc += pow((double)(i + 1), -s); cdf[i] = acc; }
    for (int i = 0; i < L; i++) cdf[i] /= acc;
    cdf[L - 1] = 2.0;
    uint64_t k = rkey(seed, 6);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) out[i] = cdf_pick(cdf, L, u01(rnd(k, (uint64_t)i)));
    free(cdf);
    return 0;
}

/* ------------------------------------------------- random-walk queries */

/* Adjacency for walking: built from the edge list by counting sort. */
typedef struct {
    int64_t n;
    int64_t* off;
    int32_t* nbr;
    uint64_t* keys;   /* sorted unordered-pair keys, for pair membership */
    int64_t nkeys;
} walk_graph;

static int pair_present(const walk_graph* g, int32_t a, int32_t b) {
    uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
    uint64_t k = (lo << 32) | hi;
    int64_t l = 0, h = g->nkeys;
    while (l < h) {
        int64_t mid = (l + h) >> 1;
        if (g->keys[mid] < k) l = mid + 1; else h = mid;
    }
    return l < g->nkeys && g->keys[l] == k;
}

/* Sorts the values a[0..n) ascending in place (LSD radix, 16-bit digits,
 * only the bits that vary; per-thread ranges as in sort_kv). */
static int sort_u64(uint64_t* a, int64_t n) {
    if (n <= 1) return 0;
    uint64_t kmax = 0;
#pragma omp parallel for reduction(| : kmax) schedule(static)
    for (int64_t i = 0; i < n; i++) kmax |= a[i];
    int bits = 0;
    while (bits < 64 && (kmax >> bits)) bits++;
    int T = omp_get_max_threads();
    if (T < 1) T = 1;
    if (T > 64) T = 64;
    if (n < (int64_t)T * 65536) T = 1;
    uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    int64_t* cnt = (int64_t*)malloc((size_t)T * 65536 * sizeof(int64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t* x = a; uint64_t* y = tmp;
    for (int sh = 0; sh < bits; sh += 16) {
        int used = T;
#pragma omp parallel num_threads(T)
        {
            const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#pragma omp single
            used = nt;
            const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* c = cnt + (int64_t)t * 65536;
            memset(c, 0, 65536 * sizeof(int64_t));
            for (int64_t i = lo; i < hi; i++) c[(x[i] >> sh) & 0xFFFF]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t s = 0;
                for (int d = 0; d < 65536; d++)
                    for (int u = 0; u < used; u++) {
                        int64_t v = cnt[(int64_t)u * 65536 + d];
                        cnt[(int64_t)u * 65536 + d] = s;
                        s += v;
                    }
            }
            for (int64_t i = lo; i < hi; i++) y[c[(x[i] >> sh) & 0xFFFF]++] = x[i];
        }
        uint64_t* t2 = x; x = y; y = t2;
    }
    if (x != a) memcpy(a, x, (size_t)n * sizeof(uint64_t));
    free(tmp); free(cnt);
    return 0;
}

void* synth_walk_graph_new(int64_t n, int64_t m, const int32_t* edges) {
    walk_graph* g = (walk_graph*)calloc(1, sizeof(walk_graph));
    if (!g) return NULL;
    g->n = n;
    g->off = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    uint64_t* key = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!g->off || !key) { free(key); free(g->off); free(g); return NULL; }
    /* distinct unordered pairs (lo << 32 | hi), ascending; loops dropped */
    int64_t nk = 0;
    for (int64_t e = 0; e < m; e++) {
        int32_t s = edges[2 * e], d = edges[2 * e + 1];
        if (s == d) continue;
        uint64_t lo = (uint64_t)(s < d ? s : d), hi = (uint64_t)(s < d ? d : s);
        key[nk++] = (lo << 32) | hi;
    }
    if (sort_u64(key, nk) != 0) { free(key); free(g->off); free(g); return NULL; }
    int64_t u = 0;
    for (int64_t i = 0; i < nk; i++)
        if (u == 0 || key[u - 1] != key[i]) key[u++] = key[i];
    g->keys = key;
    g->nkeys = u;
    /* Row v holds its smaller neighbours (pairs (lo, v), ascending lo) and
     * then its larger ones (its own run of pairs (v, hi), ascending hi): the
     * same rows a fill in key order gives.  The smaller ones come from the
     * pairs sorted by (hi, lo). */
    uint64_t* sw = (uint64_t*)malloc((size_t)(u > 0 ? u : 1) * sizeof(uint64_t));
    int64_t* nlo = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));   /* pairs with lo = v */
    int64_t* nhi = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));   /* pairs with hi = v */
    if (!sw || !nlo || !nhi) { free(sw); free(nlo); free(nhi); free(key); free(g->off); free(g); return NULL; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < u; i++) sw[i] = (key[i] << 32) | (key[i] >> 32);
    if (sort_u64(sw, u) != 0) { free(sw); free(nlo); free(nhi); free(key); free(g->off); free(g); return NULL; }
    for (int64_t i = 0; i < u; i++) { nlo[key[i] >> 32]++; nhi[sw[i] >> 32]++; }
    /* offsets, and where each row's run starts in key[] and in sw[] */
    int64_t* slo = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t* shi = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!slo || !shi) { free(slo); free(shi); free(sw); free(nlo); free(nhi); free(key); free(g->off); free(g); return NULL; }
    int64_t ol = 0, oh = 0;
    for (int64_t v = 0; v < n; v++) {
        slo[v] = ol; shi[v] = oh;
        ol += nlo[v]; oh += nhi[v];
        g->off[v + 1] = g->off[v] + nlo[v] + nhi[v];
    }
    g->nbr = (int32_t*)malloc((size_t)(g->off[n] > 0 ? g->off[n] : 1) * sizeof(int32_t));
    if (!g->nbr) { free(slo); free(shi); free(sw); free(nlo); free(nhi); free(key); free(g->off); free(g); return NULL; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < u; i++) {
        int64_t v = (int64_t)(sw[i] >> 32);                        /* pair (lo, v): v's smaller neighbour */
        g->nbr[g->off[v] + (i - shi[v])] = (int32_t)(sw[i] & 0xFFFFFFFFu);
        int64_t w = (int64_t)(key[i] >> 32);                       /* pair (w, hi): w's larger neighbour */
        g->nbr[g->off[w] + nhi[w] + (i - slo[w])] = (int32_t)(key[i] & 0xFFFFFFFFu);
    }
    free(slo); free(shi); free(sw); free(nlo); free(nhi);
    return g;
}

void synth_walk_graph_free(void* p) {
    walk_graph* g = (walk_graph*)p;
    if (!g) return;
    free(g->off); free(g->nbr); free(g->keys); free(g);
}

/*
 * One query of k vertices from a simple random walk on G.
 *   kind 0 ("induced"): every G edge among the walk's vertices.
 *   kind 1 ("dense"):   as kind 0, accepted only when 2|E|/k > 3.
 *   kind 2 ("sparse"):  the walk's first-visit tree edges plus a random
 *                       subset of the other induced edges, |E| <= 1.5k
 *                       (average degree <= 3).
 * Query vertex i is the i-th distinct vertex the walk visits, labelled as in
 * G, so the identity (query vertex i -> verts_out[i]) is always a match.
 * Returns the edge count (>= k-1), or a negative code when no walk from
 * max_attempts starts succeeds.
 */
int synth_walk_query(const void* gp, const int32_t* labels, int k, int kind, uint64_t seed,
                     uint64_t stream, int max_attempts, int32_t* verts_out,
                     int32_t* qlabels_out, int32_t* qedges_out /*[k*(k-1)/2][2]*/) {
    const walk_graph* g = (const walk_graph*)gp;
    if (k < 1 || k > 64) return -4;
    uint64_t key = rkey(seed, 1000003ull + stream);
    uint64_t ctr = 0;
    int32_t tree_a[64], tree_b[64];
    int32_t ea[2080], eb[2080];
    for (int att = 0; att < max_attempts; att++) {
        int32_t cur = (int32_t)below(rnd(key, ctr++), (uint64_t)g->n);
        int nv = 1;
        verts_out[0] = cur;
        int ok = 1;
        long steps = 0, max_steps = 200L * k + 1000;
        while (nv < k) {
            int64_t d = g->off[cur + 1] - g->off[cur];
            if (d == 0 || steps++ > max_steps) { ok = 0; break; }
            int32_t nx = g->nbr[g->off[cur] + (int64_t)below(rnd(key, ctr++), (uint64_t)d)];
            int seen = 0;
            for (int i = 0; i < nv; i++) if (verts_out[i] == nx) { seen = 1; break; }
            if (!seen) {
                int pi = 0;
                for (int i = 0; i < nv; i++) if (verts_out[i] == cur) { pi = i; break; }
                tree_a[nv - 1] = pi; tree_b[nv - 1] = nv;
                verts_out[nv++] = nx;
            }
            cur = nx;
        }
        if (!ok) continue;
        int ne = 0;
        for (int i = 0; i < k; i++)
            for (int j = i + 1; j < k; j++)
                if (pair_present(g, verts_out[i], verts_out[j])) { ea[ne] = i; eb[ne] = j; ne++; }
        if (kind == 1 && !(2 * ne > 3 * k)) continue;
        for (int i = 0; i < k; i++) qlabels_out[i] = labels[verts_out[i]];
        if (kind == 0 || kind == 1) {
            for (int e = 0; e < ne; e++) { qedges_out[2 * e] = ea[e]; qedges_out[2 * e + 1] = eb[e]; }
            return ne;
        }
        /* sparse: tree edges first, then shuffled extras up to 1.5k edges */
        int out = 0;
        for (int t = 0; t < k - 1; t++) { qedges_out[2 * out] = tree_a[t]; qedges_out[2 * out + 1] = tree_b[t]; out++; }
        int32_t xa[2080], xb[2080];
        int nx = 0;
        for (int e = 0; e < ne; e++) {
            int is_tree = 0;
            for (int t = 0; t < k - 1; t++)
                if ((tree_a[t] == ea[e] && tree_b[t] == eb[e]) || (tree_a[t] == eb[e] && tree_b[t] == ea[e])) { is_tree = 1; break; }
            if (!is_tree) { xa[nx] = ea[e]; xb[nx] = eb[e]; nx++; }
        }
        for (int i = nx - 1; i > 0; i--) {
            int j = (int)below(rnd(key, ctr++), (uint64_t)(i + 1));
            int32_t t = xa[i]; xa[i] = xa[j]; xa[j] = t;
            t = xb[i]; xb[i] = xb[j]; xb[j] = t;
        }
        int cap = (3 * k) / 2;
        for (int i = 0; i < nx && out < cap; i++) { qedges_out[2 * out] = xa[i]; qedges_out[2 * out + 1] = xb[i]; out++; }
        return out;
    }
    return -5;
}
