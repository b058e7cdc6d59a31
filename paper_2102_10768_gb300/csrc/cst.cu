// Candidate search tree construction (Sec. IV-A, Algorithm 1) and the
// workload estimate (Sec. IV-C), on the device.
//
// Steps (each a handful of kernels; the host only sequences them and reads
// candidate counts, which decide the root and the matching order):
//   filter     |C0(u)| for every u in one launch over the label buckets.
//   top-down   per tree edge (u_p -> u): the neighbour lists of C(u_p) -- only
//              their run of u's label when the graph groups rows by label -- are
//              flattened into one edge space (prefix sum of their lengths); an
//              ordered compaction keeps neighbours that pass u's filter,
//              writing N^{u_p}_u(v_p) in place and marking the reached
//              vertices in a bitmap, whose compaction is C(u).
//   bottom-up  per u, children first: a pass over each child's flattened
//              lists flags the candidates that keep an entry alive in the
//              child's bitmap; candidates with an empty child list are
//              dropped; an ordered compaction rewrites the surviving lists as
//              candidate-local indices (bitmap rank).
//   non-tree   per non-tree edge (earlier u_j -> later u_i in the order):
//              the same edge-space compaction over C(u_j) with the bitmap of
//              C(u_i) as predicate and its rank as output.
//   workload   children first: the saturating sum of c over each child
//              list (entry-parallel, one atomic per row segment), then their
//              product per candidate.
// Buffers are sized by host-known bounds and taken from the scratch pool;
// the last round trip gives every exact size, and one kernel copies the
// CST's arrays into one exact-size block that the CST owns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "prims.cuh"
#include "seg.cuh"
#include "cst_funcs.cuh"

using namespace fast;

namespace {

// ------------------------------------------------------------ small kernels

__global__ void k_filter_count(const int32_t* __restrict__ lab_vtx, const int32_t* __restrict__ key,
                               const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                               const int32_t* __restrict__ dq, unsigned long long* __restrict__ cnt) {
    int u = blockIdx.y;
    int64_t a = lo[u], b = hi[u];
    int want = dq[u];
    unsigned long long c = 0;
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x)
        c += ((key[lab_vtx[i]] & 255) >= want) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt[u], c);
}

// Label-frequency filter (filter_rule 1).  For every query vertex u
// (blockIdx.y) and every vertex v of u's label bucket: v passes if
// d(v) >= d_q(u) and, for each label that n_u of u's query neighbours carry,
// v has at least n_u neighbours with that label (its label run, or a count
// along the row when the graph is not grouped).  Passing vertices get a bit
// in u's bitmap; cnt[u] counts them.

__global__ void k_filter_nlf(const int32_t* __restrict__ lab_vtx, const int32_t* __restrict__ key,
                             const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                             const int32_t* __restrict__ dq, const __grid_constant__ NlfReq R, GraphRuns G,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ label,
                             uint32_t* __restrict__ bits, int64_t nw, unsigned long long* __restrict__ cnt) {
    const int u = blockIdx.y;
    const int64_t a = lo[u], b = hi[u];
    const int want = dq[u];
    uint32_t* bu = bits + (int64_t)u * nw;
    unsigned long long c = 0;
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = lab_vtx[i];
        bool ok = (key[v] & 255) >= want;
        for (int t = 0; ok && t < R.nn[u]; t++)
            ok = neighbours_with_label(G, col, label, v, R.lab[u][t]) >= R.need[u][t];
        if (ok) {
            atomicOr(&bu[v >> 5], 1u << (v & 31));
            c++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt[u], c);
}

// Per candidate row: where its neighbours with label l start in col (beg)
// and how many there are (len) -- the label's run of a grouped graph, or the
// whole row otherwise.
__global__ void k_cand_segment(const int32_t* __restrict__ cand, int64_t nc, GraphRuns G, int32_t l,
                               int64_t* __restrict__ beg, int64_t* __restrict__ len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) label_segment(G, cand[i], l, beg + i, len + i);
}

// the same for the first *n candidates, zero length up to the bound `cap`
__global__ void k_cand_segment_n(const int32_t* __restrict__ cand, const int64_t* __restrict__ n, int64_t cap,
                                 GraphRuns G, int32_t l, int64_t* __restrict__ beg, int64_t* __restrict__ len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    if (i < *n) label_segment(G, cand[i], l, beg + i, len + i);
    else { beg[i] = 0; len[i] = 0; }
}

// off[*n] = *val (closing offset of a list set whose row count is on the device)
__global__ void k_set_tail(int64_t* off, const int64_t* n, const int64_t* val) { off[*n] = *val; }

// Rows after the last entry (and the closing offset): new_off[r] = total for
// r <= n with e_off[r] == e_off[n].  n on the device (n_dev) or given.
__global__ void k_fill_tail(const int64_t* __restrict__ e_off, const int64_t* __restrict__ n_dev, int64_t n_host,
                            int64_t cap, const int64_t* __restrict__ total, int64_t* __restrict__ new_off) {
    const int64_t n = n_dev ? *n_dev : n_host;
    const int64_t end = e_off[n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n && r <= cap; r += (int64_t)gridDim.x * blockDim.x)
        if (e_off[r] == end) new_off[r] = *total;
}

__global__ void k_popc_words(const uint32_t* __restrict__ bits, int64_t nw, uint32_t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nw) out[i] = __popc(bits[i]);
}

__global__ void k_set_bits_n(const int32_t* __restrict__ ids, const int64_t* __restrict__ n, int64_t cap,
                             uint32_t* __restrict__ bits) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap && i < *n) atomicOr(&bits[ids[i] >> 5], 1u << (ids[i] & 31));
}

// ------------------------------------------------- balanced list kernels
//
// The lists of a CST level are one flattened entry space (offsets over the
// rows of a candidate set).  On a power-law graph a few hub rows hold most
// entries, so these kernels split the entry space, not the rows: a warp
// takes tiles of kWarpTileItems entries (grid-stride), finds the rows of the
// tile's ends by a 33-way search of the 32 lanes together, and each thread
// takes kItems consecutive entries, finds its first row between those two
// by binary search and advances it.

inline unsigned tile_grid(int64_t entries_bound) {
    int64_t t = ceil_div(entries_bound, (int64_t)kTileItems);
    int64_t cap = (int64_t)num_sms() * 8;
    if (t > cap) t = cap;
    return (unsigned)(t < 1 ? 1 : t);
}

// has[r] = 1 if row r (of *nrows) keeps an entry alive in `alive`.  Each
// warp takes tiles of kWarpTileItems entries (grid-stride over the warps),
// finds the rows of its first and last entries, and each thread its kItems.
__global__ void __launch_bounds__(256) k_any_alive(const int64_t* __restrict__ off, const int64_t* __restrict__ nrows,
                                                   const int32_t* __restrict__ list, const uint32_t* __restrict__ alive,
                                                   uint8_t* __restrict__ has) {
    const int64_t rows = *nrows;
    const int64_t e_end = off[rows];
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t t = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); t * kWarpTileItems < e_end;
         t += (int64_t)gridDim.x * wpb) {
        const int64_t tb = t * kWarpTileItems;
        const int64_t te = tb + kWarpTileItems < e_end ? tb + kWarpTileItems : e_end;
        int64_t r0, r1;
        warp_rows_of(off, rows, tb, te - 1, &r0, &r1);
        const int64_t i0 = tb + (int64_t)(threadIdx.x & 31) * kItems;
        if (i0 < te) {
            int64_t row = row_in(off, r0, r1, i0), done = -1;
            for (int i = 0; i < kItems; i++) {
                int64_t e = i0 + i;
                if (e >= te) break;
                while (e >= off[row + 1]) row++;
                if (row == done) continue;
                int32_t x = list[e];
                if ((alive[x >> 5] >> (x & 31)) & 1u) { has[row] = 1; done = row; }
            }
        }
        __syncwarp();
    }
}

// valid[r] = r < *nrows and every child list of row r keeps an entry
__global__ void k_valid_rows_n(ChildFlags cf, const int64_t* __restrict__ nrows, int64_t cap,
                               uint8_t* __restrict__ valid, int64_t* __restrict__ vflag) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= cap) return;
    uint8_t ok = r < *nrows ? 1 : 0;
    for (int c = 0; c < cf.nch && ok; c++) ok &= cf.has[c][r];
    valid[r] = ok;
    vflag[r] = ok;
}

// Workload, first half (Sec. IV-C): per row r of C(u) and one child c, the
// sum of c_c over r's list into c.  Warp tiles as in k_any_alive; each
// thread adds its kItems entries row by row (child_sum_entries).
__global__ void __launch_bounds__(256, 4) k_child_sums(const int64_t* __restrict__ off, int64_t rows,
                                                       const uint32_t* __restrict__ idx,
                                                       const uint64_t* __restrict__ cv, const double* __restrict__ cvf,
                                                       unsigned long long* __restrict__ ssum, double* __restrict__ sumf,
                                                       uint32_t* __restrict__ ovf) {
    const int64_t e_end = off[rows];
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t t = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); t * kWarpTileItems < e_end;
         t += (int64_t)gridDim.x * wpb) {
        const int64_t tb = t * kWarpTileItems;
        const int64_t te = tb + kWarpTileItems < e_end ? tb + kWarpTileItems : e_end;
        int64_t r0, r1;
        warp_rows_of(off, rows, tb, te - 1, &r0, &r1);
        child_sum_entries(off, r0, r1, tb + (int64_t)(threadIdx.x & 31) * kItems, te, idx, cv, cvf, ssum, sumf, ovf);
        __syncwarp();
    }
}

// Workload, second half: c_u(v) = product over children of those sums
// (saturating), and the float64 twin; the saturated sums are kept for the
// partitioner.
__global__ void k_workload_prod(ChildSums cs, int64_t rows, uint64_t* __restrict__ cval, double* __restrict__ cvalf) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    uint64_t prod = 1;
    double prodf = 1.0;
    for (int c = 0; c < cs.nch; c++) {
        uint64_t sm = cs.ovf[c][r] ? ~0ull : cs.ssum[c][r];
        cs.ssum[c][r] = sm;
        prod = sat_mul(prod, sm);
        prodf *= cs.sumf[c][r];
    }
    cval[r] = prod;
    cvalf[r] = prodf;
}

__global__ void k_total_w(const uint64_t* __restrict__ cval, const double* __restrict__ cvalf, int64_t n,
                          uint64_t* __restrict__ out, double* __restrict__ outf) {
    __shared__ uint64_t sh[32];
    __shared__ double shf[32];
    uint64_t s = 0;
    double sf = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) { s = sat_add(s, cval[i]); sf += cvalf[i]; }
    s = warp_sat_sum(s);
    sf = warp_sum_f(sf);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sh[warp] = s; shf[warp] = sf; }
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        s = lane < nw ? sh[lane] : 0;
        sf = lane < nw ? shf[lane] : 0.0;
        s = warp_sat_sum(s);
        sf = warp_sum_f(sf);
        if (lane == 0) { *out = s; *outf = sf; }
    }
}

__global__ void k_fill_u64(uint64_t* p, int64_t n, uint64_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fill_f64(double* p, int64_t n, double v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

inline unsigned grid_for(int64_t n, int threads) {
    int64_t b = ceil_div(n, threads);
    return (unsigned)(b < 1 ? 1 : (b > 0x7FFFFFFF ? 0x7FFFFFFF : b));
}

// ----------------------------------------------------------------- build

struct Bits {
    uint32_t* alive = nullptr;
    uint32_t* rank = nullptr;
};

void cst_release(fast_cst* c) {
    if (!c) return;
    c->arena.release(c->stream);
    delete c;
}

// ------------------------------------------------ exact-size CST storage

// After the last round trip every size is known: copy the CST's arrays into
// one exact-size block of its arena with one kernel.  The build buffers stay
// with the caller, who frees them.
int cst_to_arena(fast_cst* c, cudaStream_t s) {
    struct Item { void** slot; uint64_t bytes; };
    std::vector<Item> items;
    const int k = c->k;
    for (int u = 0; u < k; u++) {
        const uint64_t nc = (uint64_t)c->ncand[u];
        items.push_back({(void**)&c->cand[u], nc * 4});
        items.push_back({(void**)&c->cval[u], nc * 8});
        items.push_back({(void**)&c->cvalf[u], nc * 8});
        if (c->parent[u] >= 0) {
            const uint64_t np = (uint64_t)c->ncand[c->parent[u]];
            items.push_back({(void**)&c->t_off[u], (np + 1) * 8});
            items.push_back({(void**)&c->t_idx[u], (uint64_t)c->t_entries[u] * 4});
            items.push_back({(void**)&c->ssum[u], np * 8});
        }
    }
    for (int e = 0; e < c->nnt; e++) {
        const uint64_t nf = (uint64_t)c->ncand[c->nt_from[e]];
        items.push_back({(void**)&c->n_off[e], (nf + 1) * 8});
        items.push_back({(void**)&c->n_idx[e], (uint64_t)c->n_entries[e] * 4});
    }
    uint64_t total = 0;
    for (auto& it : items) total += (std::max<uint64_t>(it.bytes, 1) + 255) / 256 * 256;
    unsigned char* base = nullptr;
    FAST_TRY(c->arena.alloc_exact(&base, total, s));
    std::vector<CopyDesc> h;
    uint64_t at = 0, pieces = 0;
    for (auto& it : items) {
        unsigned char* dst = base + at;
        at += (std::max<uint64_t>(it.bytes, 1) + 255) / 256 * 256;
        if (it.bytes) {
            h.push_back({(const unsigned char*)*it.slot, dst, it.bytes, pieces});
            pieces += (it.bytes + kPiece - 1) / kPiece;
        }
        c->build_tmp.push_back(*it.slot);
        *it.slot = dst;
    }
    if (h.empty()) return FAST_OK;
    CopyDesc* d = nullptr;
    FAST_TRY(dalloc(&d, h.size(), s));
    FAST_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(CopyDesc), cudaMemcpyHostToDevice, s));
    unsigned grid = (unsigned)std::min<uint64_t>(pieces, (uint64_t)num_sms() * 8);
    k_copy_many<<<grid, 256, 0, s>>>(d, (int)h.size(), pieces);
    note_launch();
    int rc = cudaGetLastError() == cudaSuccess ? FAST_OK : set_error(FAST_ERR_CUDA, "CST copy launch");
    dfree(d, s);
    return rc;
}

// Frees the build's buffers of the CST arrays: those cst_to_arena replaced
// (kept in build_tmp), or, if it did not run, the arrays themselves.
void free_build_arrays(fast_cst* c, cudaStream_t s) {
    if (!c->build_tmp.empty()) {
        for (void* p : c->build_tmp) dfree(p, s);
        c->build_tmp.clear();
        return;
    }
    for (int u = 0; u < kMaxK; u++) {
        dfree(c->cand[u], s); dfree(c->t_off[u], s); dfree(c->t_idx[u], s);
        dfree(c->cval[u], s); dfree(c->cvalf[u], s); dfree(c->ssum[u], s);
    }
    for (int e = 0; e < kMaxNT; e++) { dfree(c->n_off[e], s); dfree(c->n_idx[e], s); }
}

// Lists whose upper bound exceeds this many entries are sized exactly (one
// host round trip) instead of by the bound.
constexpr int64_t kBoundedListCap = 64ll << 20;

int build_cst(const fast_graph* g, const fast_query_desc* q, const fast_config* cfg_in, cudaStream_t s,
              fast_cst** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_build_cst: out is NULL");
    *out = nullptr;
    if (!g) return set_error(FAST_ERR_INVALID, "fast_build_cst: graph is NULL");
    int A[kMaxK][kMaxK], dq[kMaxK];
    FAST_TRY(validate_query(q, A, dq));
    if (cfg_in && (cfg_in->order_rule < 0 || cfg_in->order_rule > 3))
        return set_error(FAST_ERR_INVALID, "fast_build_cst: order_rule %d (0 path-based, 1 greedy, 2 BFS, 3 fewest candidates)",
                         cfg_in->order_rule);
    if (cfg_in && (cfg_in->filter_rule < 0 || cfg_in->filter_rule > 1))
        return set_error(FAST_ERR_INVALID, "fast_build_cst: filter_rule %d (0 label and degree, 1 label frequencies)",
                         cfg_in->filter_rule);
    if (cfg_in && cfg_in->refine_rule != 0)
        return set_error(FAST_ERR_INVALID, "fast_build_cst: refine_rule %d (only fast_build_cst_batch refines further)",
                         cfg_in->refine_rule);
    const int k = q->n;
    fast_cst* c = new fast_cst();
    memset(c->cand, 0, sizeof(c->cand)); memset(c->t_off, 0, sizeof(c->t_off)); memset(c->t_idx, 0, sizeof(c->t_idx));
    memset(c->cval, 0, sizeof(c->cval)); memset(c->cvalf, 0, sizeof(c->cvalf)); memset(c->ssum, 0, sizeof(c->ssum));
    memset(c->n_off, 0, sizeof(c->n_off)); memset(c->n_idx, 0, sizeof(c->n_idx));
    memset(c->t_entries, 0, sizeof(c->t_entries)); memset(c->ncand, 0, sizeof(c->ncand));
    c->g = g; c->k = k; c->stream = s;
    if (cfg_in) c->cfg = *cfg_in; else fast_config_default(&c->cfg);
    for (int u = 0; u < k; u++) { c->qlabel[u] = q->labels[u]; c->dq[u] = dq[u]; }

    const int64_t n = g->n;
    const int64_t nw = n / 32 + 1;
    // Sizes live on the device (cnt block); buffers are sized by host-side
    // bounds: a candidate set by its label bucket, a list set by the degree
    // sum of the parent's label bucket.
    int32_t* td_list[kMaxK] = {nullptr};    // top-down lists (data-vertex ids)
    int64_t* td_off[kMaxK] = {nullptr};
    int32_t* td_cand[kMaxK] = {nullptr};    // top-down candidate sets
    int64_t cap_c[kMaxK] = {0};             // bound on |C(u)|
    int64_t cap_l[kMaxK] = {0};             // bound on the entries of the tree lists into u
    Bits bits[kMaxK];
    int64_t* e_off = nullptr;
    int64_t* seg = nullptr;                 // per candidate row: start of its label segment in col
    const GraphRuns G = graph_runs(g);
    const bool nlf = c->cfg.filter_rule == 1;
    uint32_t* nlf_bits = nullptr;           // label-frequency rule: [k][nw] bitmaps of C0
    unsigned long long* cnt_d = nullptr;
    int32_t* dq_d = nullptr;
    int64_t* lo_d = nullptr;
    // device sizes: [0,k) |C_td(u)|, [k,2k) |C(u)|, [2k,3k) tree-list entries into u,
    // [3k, 3k+nt) non-tree entries, then scratch words
    int64_t* sz = nullptr;
    const int kSzWords = 3 * kMaxK + kMaxNT + 4;
    int rc = FAST_OK;

    auto bucket = [&](int32_t l) -> int64_t {
        return (l >= 0 && l < g->num_labels) ? g->lab_ptr_host[l + 1] - g->lab_ptr_host[l] : 0;
    };
    auto degsum = [&](int32_t l) -> int64_t {
        return (l >= 0 && l < g->num_labels) ? g->lab_degsum_host[l] : 0;
    };

    do {
        rc = dalloc(&sz, kSzWords, s); if (rc) break;
        cudaMemsetAsync(sz, 0, kSzWords * sizeof(int64_t), s);
        // ---------------------------------------------------- filter counts
        int64_t lo[kMaxK], hi[kMaxK], c0[kMaxK];
        int64_t maxb = 1;
        for (int u = 0; u < k; u++) {
            int32_t l = q->labels[u];
            if (l < g->num_labels) { lo[u] = g->lab_ptr_host[l]; hi[u] = g->lab_ptr_host[l + 1]; }
            else { lo[u] = hi[u] = 0; }
            maxb = std::max<int64_t>(maxb, hi[u] - lo[u]);
            cap_c[u] = bucket(l);
        }
        rc = dalloc(&cnt_d, k, s); if (rc) break;
        rc = dalloc(&dq_d, k, s); if (rc) break;
        rc = dalloc(&lo_d, 2 * k, s); if (rc) break;
        cudaMemsetAsync(cnt_d, 0, k * sizeof(unsigned long long), s);
        cudaMemcpyAsync(dq_d, dq, k * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(lo_d, lo, k * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(lo_d + k, hi, k * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        {
            dim3 grid((unsigned)std::min<int64_t>(ceil_div(maxb, 256), 1024), (unsigned)k);
            if (nlf) {
                NlfReq R;
                memset(&R, 0, sizeof(R));
                for (int u = 0; u < k; u++)
                    for (int w = 0; w < k; w++) {
                        if (!A[u][w]) continue;
                        int t = 0;
                        while (t < R.nn[u] && R.lab[u][t] != q->labels[w]) t++;
                        if (t == R.nn[u]) { R.lab[u][t] = q->labels[w]; R.need[u][t] = 0; R.nn[u]++; }
                        R.need[u][t]++;
                    }
                rc = dalloc(&nlf_bits, (size_t)k * nw, s); if (rc) break;
                cudaMemsetAsync(nlf_bits, 0, (size_t)k * nw * sizeof(uint32_t), s);
                k_filter_nlf<<<grid, 256, 0, s>>>(g->lab_vtx, g->key, lo_d, lo_d + k, dq_d, R, G, g->col, g->label,
                                                  nlf_bits, nw, cnt_d);
            } else {
                k_filter_count<<<grid, 256, 0, s>>>(g->lab_vtx, g->key, lo_d, lo_d + k, dq_d, cnt_d);
            }
            note_launch();
        }
        unsigned long long hc[kMaxK];
        if (cudaMemcpyAsync(hc, cnt_d, k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "filter count"); break; }
        for (int u = 0; u < k; u++) c0[u] = (int64_t)hc[u];

        // ------------------------------------------------- root and t_q
        const int r = choose_root(k, c0, dq);
        c->root = r;
        bfs_tree(k, A, r, c->bfs, c->parent);
        cap_c[r] = c0[r];

        // ------------------------------------------------ C(root) = C0(root)
        rc = dalloc(&td_cand[r], cap_c[r], s); if (rc) break;
        {
            FilterF f{g->lab_vtx + lo[r], g->key, dq[r], nlf ? nlf_bits + (int64_t)r * nw : nullptr};
            rc = compact(f, hi[r] - lo[r], td_cand[r], sz + r, s); if (rc) break;
        }

        // ----------------------------------------------------- top-down
        for (int t = 1; t < k && rc == FAST_OK; t++) {
            int u = c->bfs[t], p = c->parent[u];
            int64_t rows = cap_c[p];                          // bound on |C_td(p)|
            int64_t* n_p = sz + p;                            // |C_td(p)| on the device
            rc = dalloc(&e_off, rows + 1, s); if (rc) break;
            rc = dalloc(&seg, rows, s); if (rc) break;
            if (rows > 0) {
                k_cand_segment_n<<<grid_for(rows, 256), 256, 0, s>>>(td_cand[p], n_p, rows, G, q->labels[u], seg, e_off);
                note_launch();
            }
            rc = scan_exclusive<int64_t>(e_off, e_off, rows, e_off + rows, s); if (rc) break;
            int64_t E = degsum(q->labels[p]);                 // bound on the edge space
            if (E > kBoundedListCap) {                        // too loose: size it exactly
                if (cudaMemcpyAsync(&E, e_off + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "edge space size"); break; }
            }
            cap_l[u] = E;
            rc = dalloc(&bits[u].alive, nw, s); if (rc) break;
            cudaMemsetAsync(bits[u].alive, 0, nw * sizeof(uint32_t), s);
            rc = dalloc(&td_off[u], rows + 1, s); if (rc) break;
            rc = dalloc(&td_list[u], E, s); if (rc) break;
            TopDownF f{};
            f.e_off = e_off; f.rows = rows; f.seg = seg; f.col = g->col; f.key = g->key;
            f.want_key_hi = q->labels[u]; f.want_dq = dq[u]; f.reached = bits[u].alive; f.t_off = td_off[u];
            f.label_known = G.run_ptr != nullptr;
            f.pass = nlf ? nlf_bits + (int64_t)u * nw : nullptr;
            f.E = e_off + rows;
            int64_t* kept = sz + 3 * kMaxK + kMaxNT;          // scratch word
            rc = compact(f, E, td_list[u], kept, s); if (rc) break;
            k_fill_tail<<<grid_for(rows + 1, 256), 256, 0, s>>>(e_off, n_p, 0, rows, kept, td_off[u]);
            note_launch();
            dfree(e_off, s);
            dfree(seg, s);
            rc = dalloc(&td_cand[u], cap_c[u], s); if (rc) break;
            rc = bits_ids_seg({BitsSeg{bits[u].alive, n, td_cand[u], sz + u}}, s); if (rc) break;
        }
        if (rc) break;

        // ---------------------------------------------------- bottom-up
        for (int t = k - 1; t >= 0 && rc == FAST_OK; t--) {
            int u = c->bfs[t];
            int64_t rows = cap_c[u];
            int64_t* n_u = sz + u;
            int ch[kMaxK], nch = 0;
            for (int w = 0; w < k; w++) if (c->parent[w] == u) ch[nch++] = w;
            uint8_t* has[kMaxK] = {nullptr};
            uint8_t* valid = nullptr;
            int64_t* newrow = nullptr;
            do {
                ChildFlags cf{};
                cf.nch = nch;
                for (int i = 0; i < nch; i++) {
                    int w = ch[i];
                    rc = dalloc(&has[i], rows, s); if (rc) break;
                    if (rows > 0) {
                        cudaMemsetAsync(has[i], 0, rows, s);
                        k_any_alive<<<tile_grid(cap_l[w]), 256, 0, s>>>(td_off[w], n_u, td_list[w], bits[w].alive, has[i]);
                        note_launch();
                    }
                    cf.has[i] = has[i];
                }
                if (rc) break;
                rc = dalloc(&valid, rows, s); if (rc) break;
                rc = dalloc(&newrow, rows + 1, s); if (rc) break;
                if (rows > 0) { k_valid_rows_n<<<grid_for(rows, 256), 256, 0, s>>>(cf, n_u, rows, valid, newrow); note_launch(); }
                rc = scan_exclusive<int64_t>(newrow, newrow, rows, newrow + rows, s); if (rc) break;
                rc = dalloc(&c->cand[u], rows, s); if (rc) break;
                KeepRowsF kf{td_cand[u], valid, n_u};
                rc = compact(kf, rows, c->cand[u], sz + kMaxK + u, s); if (rc) break;
                for (int i = 0; i < nch && rc == FAST_OK; i++) {
                    int w = ch[i];
                    rc = dalloc(&c->t_off[w], rows + 1, s); if (rc) break;
                    rc = dalloc(&c->t_idx[w], cap_l[w], s); if (rc) break;
                    WriteAliveF f{};
                    f.off = td_off[w]; f.nrows = n_u; f.list = td_list[w];
                    f.alive = bits[w].alive; f.rank = bits[w].rank;
                    f.valid = valid; f.newrow = newrow; f.new_off = c->t_off[w];
                    rc = compact(f, cap_l[w], c->t_idx[w], sz + 2 * kMaxK + w, s); if (rc) break;
                    k_set_tail<<<1, 1, 0, s>>>(c->t_off[w], sz + kMaxK + u, sz + 2 * kMaxK + w);
                    note_launch();
                    dfree(td_list[w], s); dfree(td_off[w], s);
                }
                if (rc) break;
                // bitmap + rank of the refined C(u)
                if (!bits[u].alive) { rc = dalloc(&bits[u].alive, nw, s); if (rc) break; }
                cudaMemsetAsync(bits[u].alive, 0, nw * sizeof(uint32_t), s);
                if (rows > 0) { k_set_bits_n<<<grid_for(rows, 256), 256, 0, s>>>(c->cand[u], sz + kMaxK + u, rows, bits[u].alive); note_launch(); }
                rc = dalloc(&bits[u].rank, nw, s); if (rc) break;
                k_popc_words<<<grid_for(nw, 256), 256, 0, s>>>(bits[u].alive, nw, bits[u].rank);
                note_launch();
                rc = scan_exclusive<uint32_t>(bits[u].rank, bits[u].rank, nw, (uint32_t*)nullptr, s);
            } while (0);
            for (int i = 0; i < nch; i++) dfree(has[i], s);
            dfree(valid, s); dfree(newrow, s);
            dfree(td_cand[u], s);
        }
        if (rc) break;
        // one round trip: the refined candidate counts decide the matching order
        {
            int64_t hs[kMaxK];
            if (cudaMemcpyAsync(hs, sz + kMaxK, k * sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "candidate counts"); break; }
            for (int u = 0; u < k; u++) c->ncand[u] = hs[u];
        }

        // ------------------------------------------------ matching order
        matching_order(k, A, r, c->parent, c->bfs, c->ncand, c->cfg.order_rule, c->order, c->pos);

        // ------------------------------------------------------ non-tree
        c->nnt = nontree_edges(k, A, c->order, c->parent, c->nt_from, c->nt_to);
        for (int e = 0; e < c->nnt && rc == FAST_OK; e++) {
            const int ui = c->nt_to[e], uj = c->nt_from[e];
            int64_t rows = c->ncand[uj];
            rc = dalloc(&e_off, rows + 1, s); if (rc) break;
            rc = dalloc(&seg, rows, s); if (rc) break;
            if (rows > 0) {
                k_cand_segment<<<grid_for(rows, 256), 256, 0, s>>>(c->cand[uj], rows, G, q->labels[ui], seg, e_off);
                note_launch();
            }
            rc = scan_exclusive<int64_t>(e_off, e_off, rows, e_off + rows, s); if (rc) break;
            int64_t E = degsum(q->labels[uj]);
            if (E > kBoundedListCap) {
                if (cudaMemcpyAsync(&E, e_off + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "edge space size"); break; }
            }
            rc = dalloc(&c->n_off[e], rows + 1, s); if (rc) break;
            rc = dalloc(&c->n_idx[e], E, s); if (rc) break;
            NonTreeF f{};
            f.e_off = e_off; f.rows = rows; f.seg = seg; f.col = g->col;
            f.alive = bits[ui].alive; f.rank = bits[ui].rank; f.n_off = c->n_off[e];
            f.E = e_off + rows;
            int64_t* kept = sz + 3 * kMaxK + e;
            rc = compact(f, E, c->n_idx[e], kept, s); if (rc) break;
            k_fill_tail<<<grid_for(rows + 1, 256), 256, 0, s>>>(e_off, nullptr, rows, rows, kept, c->n_off[e]);
            note_launch();
            dfree(e_off, s);
            dfree(seg, s);
        }
        if (rc) break;

        // ------------------------------------------------------ workload
        for (int t = k - 1; t >= 0 && rc == FAST_OK; t--) {
            int u = c->bfs[t];
            int64_t rows = c->ncand[u];
            rc = dalloc(&c->cval[u], rows, s); if (rc) break;
            rc = dalloc(&c->cvalf[u], rows, s); if (rc) break;
            ChildSums cs{};
            cs.nch = 0;
            double* sumf[kMaxK] = {nullptr};
            uint32_t* ovf[kMaxK] = {nullptr};
            for (int w = 0; w < k && rc == FAST_OK; w++) {
                if (c->parent[w] != u) continue;
                int i = cs.nch++;
                rc = dalloc(&c->ssum[w], rows, s); if (rc) break;
                rc = dalloc(&sumf[i], rows, s); if (rc) break;
                rc = dalloc(&ovf[i], rows, s); if (rc) break;
                if (rows > 0) {
                    cudaMemsetAsync(c->ssum[w], 0, rows * sizeof(uint64_t), s);
                    cudaMemsetAsync(sumf[i], 0, rows * sizeof(double), s);
                    cudaMemsetAsync(ovf[i], 0, rows * sizeof(uint32_t), s);
                    k_child_sums<<<tile_grid(cap_l[w]), 256, 0, s>>>(c->t_off[w], rows, c->t_idx[w], c->cval[w], c->cvalf[w],
                                                                   (unsigned long long*)c->ssum[w], sumf[i], ovf[i]);
                    note_launch();
                }
                cs.ssum[i] = c->ssum[w]; cs.sumf[i] = sumf[i]; cs.ovf[i] = ovf[i];
            }
            if (rc == FAST_OK && rows > 0) {
                if (cs.nch == 0) {
                    k_fill_u64<<<grid_for(rows, 256), 256, 0, s>>>(c->cval[u], rows, 1);
                    note_launch();
                    k_fill_f64<<<grid_for(rows, 256), 256, 0, s>>>(c->cvalf[u], rows, 1.0);
                    note_launch();
                } else {
                    k_workload_prod<<<grid_for(rows, 256), 256, 0, s>>>(cs, rows, c->cval[u], c->cvalf[u]);
                    note_launch();
                }
            }
            for (int i = 0; i < kMaxK; i++) { dfree(sumf[i], s); dfree(ovf[i], s); }
        }
        if (rc) break;
        {
            // the last round trip: W and every list size
            uint64_t* w_d = (uint64_t*)(sz + 3 * kMaxK + kMaxNT + 1);
            k_total_w<<<1, 1024, 0, s>>>(c->cval[r], c->cvalf[r], c->ncand[r], w_d, (double*)(w_d + 1));
            note_launch();
            int64_t hs[kSzWords];
            int lb_err = 0;
            cudaError_t e1 = cudaMemcpyAsync(hs, sz, sizeof(hs), cudaMemcpyDeviceToHost, s);
            if (e1 == cudaSuccess) e1 = cudaMemcpyFromSymbolAsync(&lb_err, g_lookback_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
            cudaError_t e2 = cudaStreamSynchronize(s);
            if (e1 != cudaSuccess || e2 != cudaSuccess) { rc = cuda_status(e2 != cudaSuccess ? e2 : e1, "fast_build_cst", __FILE__, __LINE__); break; }
            if (lb_err) { rc = set_error(FAST_ERR_CUDA, "fast_build_cst: a compaction's look-back wait ran out"); break; }
            for (int u = 0; u < k; u++) c->t_entries[u] = c->parent[u] < 0 ? 0 : hs[2 * kMaxK + u];
            for (int e = 0; e < c->nnt; e++) c->n_entries[e] = hs[3 * kMaxK + e];
            memcpy(&c->W, &hs[3 * kMaxK + kMaxNT + 1], sizeof(uint64_t));
            memcpy(&c->Wf, &hs[3 * kMaxK + kMaxNT + 2], sizeof(double));
        }
    } while (0);

    for (int u = 0; u < kMaxK; u++) {
        dfree(td_list[u], s); dfree(td_off[u], s); dfree(td_cand[u], s);
        dfree(bits[u].alive, s); dfree(bits[u].rank, s);
    }
    dfree(e_off, s); dfree(seg, s); dfree(cnt_d, s); dfree(dq_d, s); dfree(lo_d, s); dfree(sz, s);
    dfree(nlf_bits, s);
    // The lists were built in buffers sized by bounds; keep exact copies.
    if (rc == FAST_OK) rc = cst_to_arena(c, s);
    free_build_arrays(c, s);
    if (rc != FAST_OK) {
        cst_release(c);
        return rc;
    }
    *out = c;
    return FAST_OK;
}

}  // namespace

// --------------------------------------------------------------- C ABI

extern "C" int fast_build_cst(const fast_graph* g, const fast_query_desc* q, const fast_config* cfg, void* stream,
                              fast_cst** out) {
    PoolScope scratch((cudaStream_t)stream);
    return build_cst(g, q, cfg, (cudaStream_t)stream, out);
}

extern "C" int fast_cst_info(const fast_cst* c, int32_t* k, int32_t* root, int32_t* order, int32_t* parent,
                             int64_t* cand, uint64_t* w_u64, double* w_f64) {
    if (!c) return set_error(FAST_ERR_INVALID, "fast_cst_info: NULL cst");
    if (k) *k = c->k;
    if (root) *root = c->root;
    for (int i = 0; i < c->k; i++) {
        if (order) order[i] = c->order[i];
        if (parent) parent[i] = c->parent[i];
        if (cand) cand[i] = c->ncand[i];
    }
    if (w_u64) *w_u64 = c->W;
    if (w_f64) *w_f64 = c->Wf;
    return FAST_OK;
}

extern "C" int fast_cst_candidates(const fast_cst* c, int32_t u, int32_t* out, void* stream) {
    if (!c || u < 0 || u >= c->k || (!out && c->ncand[u])) return set_error(FAST_ERR_INVALID, "fast_cst_candidates: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->ncand[u]) FAST_CUDA(cudaMemcpyAsync(out, c->cand[u], c->ncand[u] * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    return FAST_OK;
}

extern "C" int fast_cst_tree_size(const fast_cst* c, int32_t u, int64_t* entries) {
    if (!c || u < 0 || u >= c->k || !entries) return set_error(FAST_ERR_INVALID, "fast_cst_tree_size: bad argument");
    *entries = c->parent[u] < 0 ? 0 : c->t_entries[u];
    return FAST_OK;
}

extern "C" int fast_cst_tree_lists(const fast_cst* c, int32_t u, int64_t* off, uint32_t* idx, void* stream) {
    if (!c || u < 0 || u >= c->k || c->parent[u] < 0 || !off || (!idx && c->t_entries[u]))
        return set_error(FAST_ERR_INVALID, "fast_cst_tree_lists: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t rows = c->ncand[c->parent[u]];
    FAST_CUDA(cudaMemcpyAsync(off, c->t_off[u], (rows + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (c->t_entries[u]) FAST_CUDA(cudaMemcpyAsync(idx, c->t_idx[u], c->t_entries[u] * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    return FAST_OK;
}

extern "C" int fast_cst_nontree_count(const fast_cst* c, int32_t* count) {
    if (!c || !count) return set_error(FAST_ERR_INVALID, "fast_cst_nontree_count: bad argument");
    *count = c->nnt;
    return FAST_OK;
}

extern "C" int fast_cst_nontree_edge(const fast_cst* c, int32_t e, int32_t* from_u, int32_t* to_u, int64_t* entries) {
    if (!c || e < 0 || e >= c->nnt) return set_error(FAST_ERR_INVALID, "fast_cst_nontree_edge: bad argument");
    if (from_u) *from_u = c->nt_from[e];
    if (to_u) *to_u = c->nt_to[e];
    if (entries) *entries = c->n_entries[e];
    return FAST_OK;
}

extern "C" int fast_cst_nontree_lists(const fast_cst* c, int32_t e, int64_t* off, uint32_t* idx, void* stream) {
    if (!c || e < 0 || e >= c->nnt || !off || (!idx && c->n_entries[e]))
        return set_error(FAST_ERR_INVALID, "fast_cst_nontree_lists: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t rows = c->ncand[c->nt_from[e]];
    FAST_CUDA(cudaMemcpyAsync(off, c->n_off[e], (rows + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (c->n_entries[e]) FAST_CUDA(cudaMemcpyAsync(idx, c->n_idx[e], c->n_entries[e] * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    return FAST_OK;
}

extern "C" int fast_cst_workload(const fast_cst* c, int32_t u, uint64_t* out, void* stream) {
    if (!c || u < 0 || u >= c->k || (!out && c->ncand[u])) return set_error(FAST_ERR_INVALID, "fast_cst_workload: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->ncand[u]) FAST_CUDA(cudaMemcpyAsync(out, c->cval[u], c->ncand[u] * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    return FAST_OK;
}

namespace fast {
void cst_release_nosync(fast_cst* c) { cst_release(c); }
}  // namespace fast

extern "C" void fast_free_cst(fast_cst* c) {
    if (!c) return;
    cudaStream_t s = c->stream;
    cst_release(c);
    cudaStreamSynchronize(s);
}
