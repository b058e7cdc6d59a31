// The CST build's compaction functors and list helpers (Sec. IV-A,
// Algorithm 1), shared by the per-query build (cst.cu) and the batched build
// (cst_batch.cu): the candidate filter, the top-down and non-tree list
// compactions, the bottom-up row selection and rewrite, the workload sums'
// child descriptors, the query check, and the exact-size copy kernel.  Each
// functor follows the compaction interface of prims.cuh (begin / eval /
// tag / at, and optionally end and counting).
#pragma once

#include "internal.cuh"
#include "prims.cuh"

namespace fast {

// C0(root): the label bucket filtered by degree (bucket order = id order)
struct FilterF {
    using value_type = int32_t;
    const int32_t* bucket;
    const int32_t* key;
    int dq;
    const uint32_t* pass;      // label-frequency rule: the vertices that passed (null: degree rule)
    __device__ void begin(int64_t) {}
    __device__ bool eval(int64_t i, int32_t& v) const {
        v = bucket[i];
        if (pass) return (pass[v >> 5] >> (v & 31)) & 1u;
        return (key[v] & 255) >= dq;
    }
    __device__ int64_t tag(int64_t) const { return -1; }
    __device__ void at(int64_t, int64_t) const {}
};

struct NlfReq {
    int nn[kMaxK];                 // distinct labels among u's query neighbours
    int32_t lab[kMaxK][kMaxK];
    int32_t need[kMaxK][kMaxK];
};

__device__ __forceinline__ int64_t neighbours_with_label(const GraphRuns& G, const int32_t* __restrict__ col,
                                                         const int32_t* __restrict__ label, int32_t v, int32_t l) {
    int64_t b, len;
    label_segment(G, v, l, &b, &len);
    if (G.run_ptr) return len;
    int64_t c = 0;                                 // ungrouped: the whole row, count it
    for (int64_t i = b; i < b + len; i++) c += label[col[i]] == l;
    return c;
}

__device__ __forceinline__ int64_t row_of(const int64_t* e_off, int64_t rows, int64_t i) {
    // last r with e_off[r] <= i
    int64_t lo = 0, hi = rows;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (e_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// row_of(e_off, rows, i) when it is known to lie in [lo, hi]
__device__ __forceinline__ int64_t row_in(const int64_t* e_off, int64_t lo, int64_t hi, int64_t i) {
    hi += 1;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (e_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// The first of the rows whose lists start at index i (row is the last one,
// the row holding entry i; the others before it are empty).
__device__ __forceinline__ int64_t first_row_at(const int64_t* e_off, int64_t row, int64_t i) {
    while (row > 0 && e_off[row - 1] == i) row--;
    return row;
}

// new_off[x] = rank for row r and every following row that starts at the
// same index (empty rows, up to the first row with an entry)
__device__ __forceinline__ void set_rows_at(const int64_t* e_off, int64_t rows, int64_t r, int64_t* new_off,
                                            int64_t rank) {
    const int64_t i = e_off[r];
    for (int64_t x = r; x < rows && e_off[x] == i; x++) new_off[x] = rank;
}

// Top-down: flattened neighbour lists of C(u_p); keeps neighbours passing
// u's filter (label and degree), marks them reached, writes list offsets.
struct TopDownF {
    using value_type = int32_t;
    const int64_t* e_off;      // [rows+1]
    int64_t rows;
    const int64_t* seg;        // per row of C(u_p): start in col of its neighbours with u's label
    const int32_t* col;
    const int32_t* key;
    int32_t want_key_hi;       // label
    int32_t want_dq;
    bool label_known;          // grouped graph: a segment holds only that label
    const uint32_t* pass;      // label-frequency rule: u's filter as a bitmap (null: label and degree)
    uint32_t* reached;         // bitmap over V(G)
    int64_t* t_off;            // out: [rows+1]
    const int64_t* E;          // edge-space size on the device (index space may be a bound)
    bool counting;             // set in the compaction's count pass: mark nothing then
    int64_t row;
    int64_t nbase;
    int64_t e_end;
    // the rows of a tile's first and last index, once per tile: each thread
    // then searches only between them
    __device__ void tile_hint(int64_t tb, int64_t te, int64_t* h) {
        const int64_t e = *E;
        if (te > e) te = e;
        int64_t r0, r1;
        warp_rows_of(e_off, rows, tb, te > tb ? te - 1 : tb, &r0, &r1);
        if ((threadIdx.x & 31) == 0) { h[0] = r0; h[1] = r1; }
    }
    __device__ void begin(int64_t i0, const int64_t* h) {
        e_end = *E;
        if (i0 >= e_end) return;
        row = row_in(e_off, h[0], h[1], i0);
        nbase = seg[row] - e_off[row];
    }
    __device__ bool eval(int64_t i, int32_t& v) {
        if (i >= e_end) { v = 0; return false; }
        while (i >= e_off[row + 1]) { row++; nbase = seg[row] - e_off[row]; }
        int32_t x = col[nbase + i];
        v = x;
        bool hit;
        if (pass) {
            hit = (pass[x >> 5] >> (x & 31)) & 1u;  // label, degree and frequencies at once
        } else if (label_known && want_dq <= 1) {
            hit = true;                        // the label is the segment's; a neighbour has degree >= 1
        } else {
            int32_t kk = key[x];
            hit = (kk >> 8) == want_key_hi && (kk & 255) >= want_dq;
        }
        if (hit && !counting) {
            // a popular vertex is reached from many rows: test the word
            // first (a stale copy only costs an atomic) and set the bit once
            const uint32_t bit = 1u << (x & 31);
            if (!(__ldcg(&reached[x >> 5]) & bit)) atomicOr(&reached[x >> 5], bit);
        }
        return hit;
    }
    // rows start at their first entry; a row with no entry (no neighbour of
    // the label) starts where the next one does, so the first entry of a
    // row tags it and every empty row just before it
    __device__ int64_t tag(int64_t i) const { return (i < e_end && i == e_off[row]) ? first_row_at(e_off, row, i) : -1; }
    // eval and tag of N consecutive indices: positions first (the row walk),
    // then every neighbour id, every filter word, every reached word at once
    template <int N>
    __device__ void eval_n(int64_t i0, int64_t end, uint32_t& keep, int32_t (&val)[N], int32_t (&tg)[N]) {
        int64_t pos[N];
#pragma unroll
        for (int j = 0; j < N; j++) {
            const int64_t i = i0 + j;
            pos[j] = -1;
            tg[j] = -1;
            if (i < end) {
                while (i >= e_off[row + 1]) { row++; nbase = seg[row] - e_off[row]; }
                pos[j] = nbase + i;
                if (i == e_off[row]) tg[j] = (int32_t)first_row_at(e_off, row, i);
            }
        }
#pragma unroll
        for (int j = 0; j < N; j++) val[j] = pos[j] >= 0 ? __ldg(col + pos[j]) : 0;
        uint32_t k = 0;
        if (pass) {
            uint32_t w[N];
#pragma unroll
            for (int j = 0; j < N; j++) w[j] = pos[j] >= 0 ? __ldg(pass + (val[j] >> 5)) : 0u;
#pragma unroll
            for (int j = 0; j < N; j++) k |= ((w[j] >> (val[j] & 31)) & 1u) << j;
        } else if (label_known && want_dq <= 1) {
#pragma unroll
            for (int j = 0; j < N; j++) k |= (pos[j] >= 0 ? 1u : 0u) << j;
        } else {
            int32_t kk[N];
#pragma unroll
            for (int j = 0; j < N; j++) kk[j] = pos[j] >= 0 ? __ldg(key + val[j]) : -1;
#pragma unroll
            for (int j = 0; j < N; j++)
                k |= ((pos[j] >= 0 && (kk[j] >> 8) == want_key_hi && (kk[j] & 255) >= want_dq) ? 1u : 0u) << j;
        }
        if (!counting) {
            uint32_t r[N];
#pragma unroll
            for (int j = 0; j < N; j++) r[j] = ((k >> j) & 1u) ? __ldcg(reached + (val[j] >> 5)) : ~0u;
#pragma unroll
            for (int j = 0; j < N; j++) {
                const uint32_t bit = 1u << (val[j] & 31);
                if (!(r[j] & bit)) atomicOr(&reached[val[j] >> 5], bit);
            }
        }
        keep = k;
    }
    __device__ void at(int64_t r, int64_t rank) const { set_rows_at(e_off, rows, r, t_off, rank); }
    __device__ int64_t end() const { return *E; }
};

// Non-tree: flattened neighbour lists of C(u_j); keeps members of C(u_i)
// (bitmap) and writes their rank in C(u_i).
struct NonTreeF {
    using value_type = uint32_t;
    const int64_t* e_off;
    int64_t rows;
    const int64_t* seg;        // per row of C(u_j): start in col of its neighbours with u_i's label
    const int32_t* col;
    const uint32_t* alive;     // bitmap of C(u_i)
    const uint32_t* rank;      // prefix popcounts of alive
    const uint2* packed;       // nullable: {alive, rank} word pairs, one 8-byte load for both
    int64_t* n_off;
    const int64_t* E;
    int64_t row;
    int64_t nbase;
    int64_t e_end;
    __device__ void tile_hint(int64_t tb, int64_t te, int64_t* h) {
        const int64_t e = *E;
        if (te > e) te = e;
        int64_t r0, r1;
        warp_rows_of(e_off, rows, tb, te > tb ? te - 1 : tb, &r0, &r1);
        if ((threadIdx.x & 31) == 0) { h[0] = r0; h[1] = r1; }
    }
    __device__ void begin(int64_t i0, const int64_t* h) {
        e_end = *E;
        if (i0 >= e_end) return;
        row = row_in(e_off, h[0], h[1], i0);
        nbase = seg[row] - e_off[row];
    }
    __device__ bool eval(int64_t i, uint32_t& v) {
        if (i >= e_end) { v = 0; return false; }
        while (i >= e_off[row + 1]) { row++; nbase = seg[row] - e_off[row]; }
        int32_t x = col[nbase + i];
        const uint2 ar = packed ? packed[x >> 5] : make_uint2(alive[x >> 5], rank[x >> 5]);
        const uint32_t bit = 1u << (x & 31);
        v = ar.y + __popc(ar.x & (bit - 1));
        return (ar.x & bit) != 0;
    }
    __device__ int64_t tag(int64_t i) const { return (i < e_end && i == e_off[row]) ? first_row_at(e_off, row, i) : -1; }
    template <int N>
    __device__ void eval_n(int64_t i0, int64_t end, uint32_t& keep, uint32_t (&val)[N], int32_t (&tg)[N]) {
        int64_t pos[N];
#pragma unroll
        for (int j = 0; j < N; j++) {
            const int64_t i = i0 + j;
            pos[j] = -1;
            tg[j] = -1;
            if (i < end) {
                while (i >= e_off[row + 1]) { row++; nbase = seg[row] - e_off[row]; }
                pos[j] = nbase + i;
                if (i == e_off[row]) tg[j] = (int32_t)first_row_at(e_off, row, i);
            }
        }
        int32_t x[N];
#pragma unroll
        for (int j = 0; j < N; j++) x[j] = pos[j] >= 0 ? __ldg(col + pos[j]) : 0;
        uint32_t w[N], rk[N];
        if (packed) {
#pragma unroll
            for (int j = 0; j < N; j++) {
                const uint2 ar = pos[j] >= 0 ? __ldg(packed + (x[j] >> 5)) : make_uint2(0u, 0u);
                w[j] = ar.x;
                rk[j] = ar.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; j++) {
                w[j] = pos[j] >= 0 ? __ldg(alive + (x[j] >> 5)) : 0u;
                rk[j] = pos[j] >= 0 ? __ldg(rank + (x[j] >> 5)) : 0u;
            }
        }
        uint32_t k = 0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            const uint32_t bit = 1u << (x[j] & 31);
            val[j] = rk[j] + __popc(w[j] & (bit - 1));
            k |= ((w[j] & bit) ? 1u : 0u) << j;
        }
        keep = k;
    }
    __device__ void at(int64_t r, int64_t rank_) const { set_rows_at(e_off, rows, r, n_off, rank_); }
    __device__ int64_t end() const { return *E; }
};

// rows kept by a validity mask
struct KeepRowsF {
    using value_type = int32_t;
    const int32_t* ids;
    const uint8_t* valid;
    const int64_t* nrows;      // rows really present (the index space is a bound)
    __device__ int64_t end() const { return *nrows; }
    __device__ void begin(int64_t) {}
    __device__ bool eval(int64_t i, int32_t& v) const {
        v = ids[i];
        return valid[i] != 0;
    }
    __device__ int64_t tag(int64_t) const { return -1; }
    __device__ void at(int64_t, int64_t) const {}
};

constexpr int kItems = 8;
constexpr int kTileItems = 256 * kItems;     // a block's tile (8 warps)
constexpr int kWarpTileItems = 32 * kItems;  // a warp's tile

// Child sums over the entries [i0, iend) of one thread (Sec. IV-C, first
// half of the workload DP: per row r and child c, the sum of c_c over r's
// list into c), rows found between r0 and r1.  A row whose entries all lie
// in the range is written with plain stores; a row shared with another
// thread is added with atomics.  Saturation: a sum that wrapped or carried a
// saturated term, or an atomic that wrapped, sets ovf[r], and the row's sum
// then reads as 2^64 - 1.
__device__ __forceinline__ void child_sum_entries(const int64_t* __restrict__ off, int64_t r0, int64_t r1, int64_t i0,
                                                  int64_t iend, const uint32_t* __restrict__ idx,
                                                  const uint64_t* __restrict__ cv, const double* __restrict__ cvf,
                                                  unsigned long long* __restrict__ ssum, double* __restrict__ sumf,
                                                  uint32_t* __restrict__ ovf) {
    if (i0 >= iend) return;
    // the thread's entries' child indices, then their values, all in flight at once
    uint32_t x[kItems];
#pragma unroll
    for (int i = 0; i < kItems; i++) x[i] = i0 + i < iend ? __ldg(idx + i0 + i) : 0u;
    uint64_t v[kItems];
    double vf[kItems];
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const bool in = i0 + i < iend;
        v[i] = in ? __ldg(cv + x[i]) : 0ull;
        vf[i] = in ? __ldg(cvf + x[i]) : 0.0;
    }
    int64_t row = row_in(off, r0, r1, i0);
    int64_t rend = off[row + 1];
    bool own = off[row] == i0;           // the row starts in this range
    unsigned long long s = 0;
    double sf = 0.0;
    bool sat = false;
    auto flush = [&](bool whole) {
        if (whole) {
            ssum[row] = s;
            sumf[row] = sf;
            if (sat) ovf[row] = 1u;
        } else {
            const unsigned long long old = atomicAdd(&ssum[row], s);
            if (old + s < old) sat = true;
            if (sat) atomicOr(&ovf[row], 1u);
            atomicAdd(&sumf[row], sf);
        }
    };
    for (int i = 0; i < kItems; i++) {
        const int64_t e = i0 + i;
        if (e >= iend) break;
        if (e >= rend) {
            flush(own);                  // the row ended inside the range
            s = 0; sf = 0.0; sat = false;
            do { row++; rend = off[row + 1]; } while (e >= rend);
            own = true;                  // a later row starts at e (empty rows between share the offset)
        }
        const unsigned long long ns = s + v[i];
        if (ns < s || v[i] == ~0ull) sat = true;
        s = ns;
        sf += vf[i];
    }
    flush(own && rend == (i0 + kItems < iend ? i0 + kItems : iend));
}

struct ChildFlags {
    const uint8_t* has[kMaxK];
    int nch;
};

// Bottom-up rewrite: the entries of valid rows still alive in the child's
// bitmap, as candidate-local indices (bitmap rank), rows renumbered by
// newrow; each kept row's new offset comes from the compaction's rank.
struct WriteAliveF {
    using value_type = uint32_t;
    const int64_t* off;
    const int64_t* nrows;
    const int32_t* list;
    const uint32_t* alive;
    const uint32_t* rank;
    const uint2* packed;       // nullable: {alive, rank} word pairs, one 8-byte load for both
    const uint8_t* valid;
    const int64_t* newrow;
    int64_t* new_off;
    int64_t rows;
    int64_t row;
    int64_t e_end;
    __device__ void tile_hint(int64_t tb, int64_t te, int64_t* h) {
        const int64_t r = *nrows, e = off[r];
        if (te > e) te = e;
        int64_t r0, r1;
        warp_rows_of(off, r, tb, te > tb ? te - 1 : tb, &r0, &r1);
        if ((threadIdx.x & 31) == 0) { h[0] = r0; h[1] = r1; }
    }
    __device__ void begin(int64_t i0, const int64_t* h) {
        rows = *nrows;
        e_end = off[rows];
        if (i0 < e_end) row = row_in(off, h[0], h[1], i0);
    }
    __device__ bool eval(int64_t i, uint32_t& v) {
        v = 0;
        if (i >= e_end) return false;
        while (i >= off[row + 1]) row++;
        if (!valid[row]) return false;
        int32_t x = list[i];
        const uint2 ar = packed ? packed[x >> 5] : make_uint2(alive[x >> 5], rank[x >> 5]);
        const uint32_t bit = 1u << (x & 31);
        v = ar.y + __popc(ar.x & (bit - 1));
        return (ar.x & bit) != 0;
    }
    __device__ int64_t tag(int64_t i) const { return (i < e_end && i == off[row] && valid[row]) ? row : -1; }
    template <int N>
    __device__ void eval_n(int64_t i0, int64_t end, uint32_t& keep, uint32_t (&val)[N], int32_t (&tg)[N]) {
        bool ok[N];
#pragma unroll
        for (int j = 0; j < N; j++) {
            const int64_t i = i0 + j;
            ok[j] = false;
            tg[j] = -1;
            if (i < end) {
                while (i >= off[row + 1]) row++;
                ok[j] = valid[row] != 0;
                if (ok[j] && i == off[row]) tg[j] = (int32_t)row;
            }
        }
        int32_t x[N];
#pragma unroll
        for (int j = 0; j < N; j++) x[j] = ok[j] ? __ldg(list + i0 + j) : 0;
        uint32_t w[N], rk[N];
        if (packed) {
#pragma unroll
            for (int j = 0; j < N; j++) {
                const uint2 ar = ok[j] ? __ldg(packed + (x[j] >> 5)) : make_uint2(0u, 0u);
                w[j] = ar.x;
                rk[j] = ar.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; j++) {
                w[j] = ok[j] ? __ldg(alive + (x[j] >> 5)) : 0u;
                rk[j] = ok[j] ? __ldg(rank + (x[j] >> 5)) : 0u;
            }
        }
        uint32_t k = 0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            const uint32_t bit = 1u << (x[j] & 31);
            val[j] = rk[j] + __popc(w[j] & (bit - 1));
            k |= ((w[j] & bit) ? 1u : 0u) << j;
        }
        keep = k;
    }
    __device__ void at(int64_t r, int64_t rk) const { new_off[newrow[r]] = rk; }
    __device__ int64_t end() const { return off[*nrows]; }
};

__device__ __forceinline__ uint64_t warp_sat_sum(uint64_t v) {
    for (int o = 16; o > 0; o >>= 1) v = sat_add(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum_f(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct ChildSums {
    uint64_t* ssum[kMaxK];
    const double* sumf[kMaxK];
    const uint32_t* ovf[kMaxK];
    int nch;
};

inline int validate_query(const fast_query_desc* q, int A[kMaxK][kMaxK], int* dq) {
    if (!q) return set_error(FAST_ERR_INVALID, "query is NULL");
    int k = q->n;
    if (k < 1 || k > kMaxK) return set_error(FAST_ERR_INVALID, "query has %d vertices (1..%d)", k, kMaxK);
    if (!q->labels || (q->m > 0 && !q->edges) || q->m < 0) return set_error(FAST_ERR_INVALID, "query arrays are NULL");
    memset(A, 0, sizeof(int) * kMaxK * kMaxK);
    for (int u = 0; u < k; u++) {
        dq[u] = 0;
        if (q->labels[u] < 0) return set_error(FAST_ERR_INVALID, "query label < 0");
    }
    for (int e = 0; e < q->m; e++) {
        int a = q->edges[2 * e], b = q->edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k) return set_error(FAST_ERR_INVALID, "query edge (%d,%d) out of range", a, b);
        if (a == b) return set_error(FAST_ERR_INVALID, "query edge (%d,%d) is a loop", a, b);
        if (!A[a][b]) { A[a][b] = A[b][a] = 1; dq[a]++; dq[b]++; }
    }
    // connected?
    int seen[kMaxK] = {0}, st[kMaxK], sp = 0, cnt = 1;
    st[sp++] = 0; seen[0] = 1;
    while (sp) {
        int u = st[--sp];
        for (int w = 0; w < k; w++) if (A[u][w] && !seen[w]) { seen[w] = 1; st[sp++] = w; cnt++; }
    }
    if (cnt != k) return set_error(FAST_ERR_INVALID, "query graph is disconnected");
    return FAST_OK;
}

// ---------------------------------------------------------------------------
// Host rules of query preparation, shared by the per-query and the batched
// builds (Sec. IV-A and IV-B; the tie-breaks the paper leaves open are fixed
// here once).

// Root of t_q: argmin |C0(u)| / d_q(u), compared exactly by cross
// multiplication; ties go to the smaller id.
inline int choose_root(int k, const int64_t* c0, const int* dq) {
    int r = 0;
    for (int u = 1; u < k; u++)
        if ((unsigned __int128)c0[u] * (unsigned)dq[r] < (unsigned __int128)c0[r] * (unsigned)dq[u]) r = u;
    return r;
}

// BFS tree t_q from r, neighbours visited in increasing id: bfs[] is the
// visiting order, parent[r] = -1.
inline void bfs_tree(int k, const int A[kMaxK][kMaxK], int r, int* bfs, int* parent) {
    int seen[kMaxK] = {0}, qh = 0, qt = 0;
    bfs[qt++] = r;
    seen[r] = 1;
    parent[r] = -1;
    while (qh < qt) {
        const int u = bfs[qh++];
        for (int w = 0; w < k; w++)
            if (A[u][w] && !seen[w]) { seen[w] = 1; parent[w] = u; bfs[qt++] = w; }
    }
}

// Matching order from the refined candidate counts.  rule 0 (path-based):
// depth-first preorder of t_q, children by increasing (|C|, id), so whole
// root-to-leaf paths come in turn.  rule 1 (greedy): after the root, the
// unplaced vertex whose t_q parent is placed with the most query edges to
// placed vertices; ties to the smaller |C|, then the smaller id.  rule 2:
// the BFS order of t_q (bfs[]).  rule 3: after the root, the unplaced
// vertex whose t_q parent is placed with the fewest candidates; ties to the
// smaller id.  Every rule places a vertex after its t_q parent.  Writes
// order[position] and pos[vertex].
inline void matching_order(int k, const int A[kMaxK][kMaxK], int r, const int* parent, const int* bfs,
                           const int64_t* ncand, int rule, int* order, int* pos) {
    if (rule == 2) {
        for (int i = 0; i < k; i++) order[i] = bfs[i];
    } else if (rule == 3) {
        bool placed[kMaxK] = {false};
        order[0] = r;
        placed[r] = true;
        for (int no = 1; no < k; no++) {
            int best = -1;
            for (int u = 0; u < k; u++) {
                if (placed[u] || !placed[parent[u]]) continue;
                if (best < 0 || ncand[u] < ncand[best] || (ncand[u] == ncand[best] && u < best)) best = u;
            }
            order[no] = best;
            placed[best] = true;
        }
    } else if (rule == 1) {
        bool placed[kMaxK] = {false};
        order[0] = r;
        placed[r] = true;
        for (int no = 1; no < k; no++) {
            int best = -1, bb = -1;
            for (int u = 0; u < k; u++) {
                if (placed[u] || !placed[parent[u]]) continue;
                int b = 0;
                for (int w = 0; w < k; w++) b += (placed[w] && A[u][w]) ? 1 : 0;
                if (best < 0 || b > bb || (b == bb && (ncand[u] < ncand[best] || (ncand[u] == ncand[best] && u < best)))) {
                    best = u;
                    bb = b;
                }
            }
            order[no] = best;
            placed[best] = true;
        }
    } else {
        int stack[kMaxK], sp = 0, no = 0;
        stack[sp++] = r;
        while (sp) {
            const int u = stack[--sp];
            order[no++] = u;
            int chl[kMaxK], nc = 0;
            for (int w = 0; w < k; w++) if (parent[w] == u) chl[nc++] = w;
            for (int i = 1; i < nc; i++)                  // insertion sort by (|C|, id)
                for (int j = i; j > 0; j--) {
                    const int a = chl[j - 1], b = chl[j];
                    if (ncand[b] < ncand[a] || (ncand[b] == ncand[a] && b < a)) { chl[j - 1] = b; chl[j] = a; }
                    else break;
                }
            for (int i = nc - 1; i >= 0; i--) stack[sp++] = chl[i];
        }
    }
    for (int i = 0; i < k; i++) pos[order[i]] = i;
}

// Non-tree edges of q, each once, from the earlier to the later endpoint in
// the order, listed by the later endpoint's position, then the earlier's.
// Returns their number.
inline int nontree_edges(int k, const int A[kMaxK][kMaxK], const int* order, const int* parent, int* from, int* to) {
    int n = 0;
    for (int i = 0; i < k; i++) {
        const int ui = order[i];
        for (int j = 0; j < i; j++) {
            const int uj = order[j];
            if (!A[ui][uj] || parent[ui] == uj || parent[uj] == ui) continue;
            from[n] = uj;
            to[n] = ui;
            n++;
        }
    }
    return n;
}

// One flat copy list: descriptor d moves bytes [0, n_d) from src_d to dst_d;
// piece_off[d] is the first 64 KB piece of d in a flat piece space.
struct CopyDesc {
    const unsigned char* src;
    unsigned char* dst;
    uint64_t bytes;
    uint64_t piece_off;
};
constexpr uint64_t kPiece = 64 << 10;

static __global__ void k_copy_many(const CopyDesc* __restrict__ d, int nd, uint64_t npieces) {
    for (uint64_t p = blockIdx.x; p < npieces; p += gridDim.x) {
        int lo = 0, hi = nd;                                  // last d with piece_off <= p
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (d[mid].piece_off <= p) lo = mid; else hi = mid;
        }
        const CopyDesc& c = d[lo];
        uint64_t a = (p - c.piece_off) * kPiece, b = a + kPiece < c.bytes ? a + kPiece : c.bytes;
        // both ends are 256-byte aligned and a is a multiple of kPiece: 16-byte words, then a byte tail
        uint64_t a16 = a / 16, b16 = b / 16;
        const uint4* s4 = (const uint4*)c.src;
        uint4* d4 = (uint4*)c.dst;
        for (uint64_t i = a16 + threadIdx.x; i < b16; i += blockDim.x) d4[i] = s4[i];
        for (uint64_t i = b16 * 16 + threadIdx.x; i < b; i += blockDim.x) c.dst[i] = c.src[i];
    }
}

}  // namespace fast
