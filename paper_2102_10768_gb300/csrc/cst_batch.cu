// Batched CST construction: the candidate search trees (Sec. IV-A,
// Algorithm 1) and workload estimates (Sec. IV-C) of many queries built
// together.
//
// The per-query build (cst.cu) runs each query's steps as launches of their
// own, with host round trips in between; for hundreds of queries the host
// side of those launches and synchronisations dominates.  Here the steps go
// over BFS positions t = 0, 1, ...: the vertex at position t of every query
// is handled by one launch per step for the whole batch (each query, or
// query edge, is one segment of a segmented compaction or scan, or a range
// of items of a plain kernel), and the host reads sizes back once or twice
// per position for all queries at once.  Each step applies the same
// functors (cst_funcs.cuh) to the same inputs as the per-query build, so
// every array of every CST comes out identical.  Buffers are sized exactly
// from those round trips and carved from a few scratch blocks per step.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "cst_funcs.cuh"
#include "internal.cuh"
#include "seg.cuh"

using namespace fast;

namespace {

// ------------------------------------------------------------- kernels

// fn(s, i) for every item i < n_s of every segment s; the items of all
// segments lie end to end (segment s starts at item_off[s]).
template <class Fn>
__device__ __forceinline__ void for_items(const int64_t* __restrict__ item_off, int nseg, Fn fn) {
    const int64_t total = item_off[nseg];
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int s = seg_of_tile(item_off, nseg, gi);
        fn(s, gi - item_off[s]);
    }
}

inline unsigned items_grid(int64_t total) {
    int64_t b = ceil_div(total, 256);
    int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// Label-frequency requirement of one query vertex u: for each of the nn
// distinct labels among u's query neighbours, how many carry it.
struct NlfRow {
    int nn;
    int32_t lab[kMaxK];
    int32_t need[kMaxK];
};

// One (query, vertex) pair of the candidate filter: the vertex's label
// bucket lab_vtx[lo, hi), its query degree and, under the label-frequency
// rule, its requirement and pass bitmap.
struct FilterDesc {
    int64_t lo, hi;
    int32_t dq;
    int32_t nlf;
    NlfRow r;
    uint32_t* bits;
    unsigned long long* cnt;
};

// |C0(u)| for every pair (blockIdx.y) in one launch: the label-and-degree
// count of k_filter_count, or the label-frequency test and bitmap of
// k_filter_nlf, per pair.
__global__ void k_filter_b(const FilterDesc* __restrict__ D, const int32_t* __restrict__ lab_vtx,
                           const int32_t* __restrict__ key, GraphRuns G, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ label) {
    const FilterDesc& d = D[blockIdx.y];
    const int64_t a = d.lo, b = d.hi;
    const int want = d.dq;
    unsigned long long c = 0;
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = lab_vtx[i];
        bool ok = (key[v] & 255) >= want;
        if (d.nlf) {
            for (int t = 0; ok && t < d.r.nn; t++)
                ok = neighbours_with_label(G, col, label, v, d.r.lab[t]) >= d.r.need[t];
            if (ok) atomicOr(&d.bits[v >> 5], 1u << (v & 31));
        }
        c += ok ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(d.cnt, c);
}

// Label segments of a candidate set's rows (as k_cand_segment): n rows, and
// one more item that zeroes len[n], so that an exclusive scan of n + 1
// lengths leaves the edge-space size in len[n].
struct CandSegDesc {
    const int32_t* cand;
    int64_t n;                       // rows (a bound when n_dev is set)
    const int64_t* n_dev;            // device, nullable: the real rows
    int32_t l;
    int64_t* beg;
    int64_t* len;
};

__global__ void k_cand_segment_b(const CandSegDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg,
                                 GraphRuns G) {
    for_items(item_off, nseg, [&](int s, int64_t i) {
        const CandSegDesc& d = D[s];
        const int64_t n = d.n_dev ? *d.n_dev : d.n;
        if (i < n) label_segment(G, d.cand[i], d.l, d.beg + i, d.len + i);
        else d.len[i] = 0;
    });
}

// Rows after the last entry and the closing offset (as k_fill_tail).
struct FillTailDesc {
    const int64_t* e_off;
    int64_t n;                       // rows
    const int64_t* total;            // device: entries kept
    int64_t* new_off;
};

__global__ void k_fill_tail_b(const FillTailDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg) {
    for_items(item_off, nseg, [&](int s, int64_t r) {
        const FillTailDesc& d = D[s];
        if (d.e_off[r] == d.e_off[d.n]) d.new_off[r] = *d.total;
    });
}

// has[r] = 1 if row r keeps an entry alive (as k_any_alive), tiles of all
// (query, child) pairs in one sequence.
struct AnyAliveDesc {
    const int64_t* off;
    int64_t rows;
    const int32_t* list;
    const uint32_t* alive;
    uint8_t* has;
};

// A warp's tile t of a tile-split batched step: its segment, its entries
// [tb, te) and the rows r0, r1 of its first and last entries, found by the
// 32 lanes together (every lane returns them).
struct WarpTile {
    int s;
    int64_t tb, te, r0, r1;
};

template <class D>
__device__ __forceinline__ WarpTile warp_tile(const D* __restrict__ Dd, const int64_t* __restrict__ tile_off, int nseg,
                                              int64_t t) {
    WarpTile w;
    w.s = seg_of_tile(tile_off, nseg, t);
    const D& d = Dd[w.s];
    const int64_t e_end = d.off[d.rows];
    w.tb = (t - tile_off[w.s]) * kWarpTileItems;
    w.te = w.tb + kWarpTileItems < e_end ? w.tb + kWarpTileItems : e_end;
    w.r0 = w.r1 = 0;
    if (w.tb < w.te) warp_rows_of(d.off, d.rows, w.tb, w.te - 1, &w.r0, &w.r1);
    return w;
}

// grid-stride over the warps of the grid
#define FOR_WARP_TILES(t, total)                                                                        \
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < (total);       \
         t += (int64_t)gridDim.x * (blockDim.x >> 5))

// A block's tile t (kTileItems entries): warp 0 finds its segment and the
// rows of its first and last entries, the block waits for them.
struct TileRows {
    int s;
    int64_t tb, te, r0, r1;
};

template <class D>
__device__ __forceinline__ bool tile_rows(const D* __restrict__ Dd, const int64_t* __restrict__ tile_off, int nseg,
                                          int64_t t, TileRows* sh) {
    if (threadIdx.x < 32) {
        const int s = seg_of_tile(tile_off, nseg, t);
        const D& d = Dd[s];
        const int64_t e_end = d.off[d.rows];
        const int64_t tb = (t - tile_off[s]) * kTileItems;
        const int64_t te = tb + kTileItems < e_end ? tb + kTileItems : e_end;
        int64_t r0 = 0, r1 = 0;
        if (tb < te) {                  // one search after the other: 32 registers, 8 blocks per SM
            r0 = warp_row_of(d.off, d.rows, tb);
            r1 = warp_row_of(d.off, d.rows, te - 1);
        }
        if (threadIdx.x == 0) { sh->s = s; sh->tb = tb; sh->te = te; sh->r0 = r0; sh->r1 = r1; }
    }
    __syncthreads();
    return sh->tb < sh->te;
}

// Block tiles here: the per-entry work (one list entry, one bitmap word) is
// small next to a row search per warp tile.
__global__ void __launch_bounds__(256) k_any_alive_b(const AnyAliveDesc* __restrict__ D,
                                                     const int64_t* __restrict__ tile_off, int nseg) {
    __shared__ TileRows tr;
    const int64_t total = tile_off[nseg];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        if (tile_rows(D, tile_off, nseg, t, &tr)) {
            const AnyAliveDesc& d = D[tr.s];
            const int64_t* off = d.off;
            const int64_t i0 = tr.tb + (int64_t)threadIdx.x * kItems;
            if (i0 < tr.te) {
                int64_t row = row_in(off, tr.r0, tr.r1, i0), done = -1;
                for (int i = 0; i < kItems; i++) {
                    int64_t e = i0 + i;
                    if (e >= tr.te) break;
                    while (e >= off[row + 1]) row++;
                    if (row == done) continue;
                    int32_t x = d.list[e];
                    if ((d.alive[x >> 5] >> (x & 31)) & 1u) { d.has[row] = 1; done = row; }
                }
            }
        }
        __syncthreads();
    }
}

// {alive, rank} word pairs of a refined candidate bitmap, so that the
// bottom-up rewrite and the non-tree step read a word and its prefix
// popcount with one 8-byte load.
struct PackDesc {
    const uint32_t* alive;
    const uint32_t* rank;
    uint2* packed;
};

__global__ void k_pack_bits_b(const PackDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg) {
    for_items(item_off, nseg, [&](int s, int64_t w) {
        const PackDesc& d = D[s];
        d.packed[w] = make_uint2(d.alive[w], d.rank[w]);
    });
}

// valid[r] = every child list of row r keeps an entry (as k_valid_rows_n).
struct ValidDesc {
    ChildFlags cf;
    uint8_t* valid;
    int64_t* vflag;
};

__global__ void k_valid_rows_b(const ValidDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg) {
    for_items(item_off, nseg, [&](int s, int64_t r) {
        const ValidDesc& d = D[s];
        uint8_t ok = 1;
        for (int c = 0; c < d.cf.nch && ok; c++) ok &= d.cf.has[c][r];
        d.valid[r] = ok;
        d.vflag[r] = ok;
    });
}

// Refine rule 2, the non-tree test: flag[r] = 1 if candidate cand[r] of u
// has a neighbour in the bitmap of C(w), for one non-tree query neighbour w
// (its label segment in G; every member of the bitmap carries w's label, so
// an ungrouped row needs no label test).  One warp per row, rows of all
// (query, neighbour) pairs end to end.
struct NtDesc {
    const int32_t* cand;
    int32_t l;
    const uint32_t* bits;
    uint8_t* flag;
};

__global__ void k_nt_support_b(const NtDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg,
                               GraphRuns G, const int32_t* __restrict__ col) {
    const int lane = threadIdx.x & 31;
    const int64_t total = item_off[nseg];
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < total;
         it += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int s = seg_of_tile(item_off, nseg, it);
        const NtDesc& d = D[s];
        const int64_t r = it - item_off[s];
        int64_t b, len;
        label_segment(G, d.cand[r], d.l, &b, &len);
        bool any = false;
        for (int64_t base = 0; base < len; base += 32) {      // the same steps on every lane
            bool hit = false;
            if (base + lane < len) {
                const int32_t x = col[b + base + lane];
                hit = (d.bits[x >> 5] >> (x & 31)) & 1u;
            }
            if (__any_sync(0xffffffffu, hit)) { any = true; break; }
        }
        if (lane == 0) d.flag[r] = any ? 1 : 0;
    }
}

// off[*n] = *val (as k_set_tail), one thread per descriptor.
struct SetTailDesc {
    int64_t* off;
    const int64_t* n;
    const int64_t* val;
};

__global__ void k_set_tail_b(const SetTailDesc* __restrict__ D, int nd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nd) D[i].off[*D[i].n] = *D[i].val;
}

// Bitmap of a candidate set whose size *n is on the device (as
// k_set_bits_n); the items of a segment are a host bound on *n.
struct SetBitsDesc {
    const int32_t* ids;
    const int64_t* n;
    uint32_t* bits;
};

__global__ void k_set_bits_b(const SetBitsDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg) {
    for_items(item_off, nseg, [&](int s, int64_t i) {
        const SetBitsDesc& d = D[s];
        if (i < *d.n) atomicOr(&d.bits[d.ids[i] >> 5], 1u << (d.ids[i] & 31));
    });
}

// Workload, first half (as k_child_sums), tiles of all (query, child)
// pairs in one sequence.
struct ChildSumDesc {
    const int64_t* off;
    int64_t rows;
    const uint32_t* idx;
    const uint64_t* cv;
    const double* cvf;
    unsigned long long* ssum;
    double* sumf;
    uint32_t* ovf;
};

__global__ void __launch_bounds__(256, 4) k_child_sums_b(const ChildSumDesc* __restrict__ D,
                                                         const int64_t* __restrict__ tile_off, int nseg) {
    const int64_t total = tile_off[nseg];
    FOR_WARP_TILES(t, total) {
        const WarpTile w = warp_tile(D, tile_off, nseg, t);
        const ChildSumDesc& d = D[w.s];
        child_sum_entries(d.off, w.r0, w.r1, w.tb + (int64_t)(threadIdx.x & 31) * kItems, w.te, d.idx, d.cv, d.cvf,
                          d.ssum, d.sumf, d.ovf);
        __syncwarp();
    }
}

// Workload, second half (as k_workload_prod; a leaf, with no child, gets
// 1 and 1.0 as k_fill_u64 / k_fill_f64 give it).
struct ProdDesc {
    ChildSums cs;
    uint64_t* cval;
    double* cvalf;
};

__global__ void k_workload_prod_b(const ProdDesc* __restrict__ D, const int64_t* __restrict__ item_off, int nseg) {
    for_items(item_off, nseg, [&](int s, int64_t r) {
        const ProdDesc& d = D[s];
        uint64_t prod = 1;
        double prodf = 1.0;
        for (int c = 0; c < d.cs.nch; c++) {
            uint64_t sm = d.cs.ovf[c][r] ? ~0ull : d.cs.ssum[c][r];
            d.cs.ssum[c][r] = sm;
            prod = sat_mul(prod, sm);
            prodf *= d.cs.sumf[c][r];
        }
        d.cval[r] = prod;
        d.cvalf[r] = prodf;
    });
}

// W per query (as k_total_w), one block of 1024 threads per descriptor.
struct TotalDesc {
    const uint64_t* cval;
    const double* cvalf;
    int64_t n;
    uint64_t* out;
    double* outf;
};

__global__ void k_total_w_b(const TotalDesc* __restrict__ D) {
    __shared__ uint64_t sh[32];
    __shared__ double shf[32];
    const TotalDesc& d = D[blockIdx.x];
    uint64_t s = 0;
    double sf = 0.0;
    for (int64_t i = threadIdx.x; i < d.n; i += blockDim.x) { s = sat_add(s, d.cval[i]); sf += d.cvalf[i]; }
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
        if (lane == 0) { *d.out = s; *d.outf = sf; }
    }
}

// ------------------------------------------------------------ host side

// Scratch blocks of one scope, returned to the pool when it ends (the pool
// only reuses them for work ordered after it on the same stream).
struct Scratch {
    explicit Scratch(cudaStream_t s) : s_(s) {}
    ~Scratch() { release(); }
    void release() {
        for (auto& p : v) dfree(p, s_);
        v.clear();
    }
    std::vector<unsigned char*> v;
    cudaStream_t s_;
};

// Arrays allocated together as one block of 256-byte aligned pieces.
class Carver {
  public:
    template <class T>
    void add(T** slot, int64_t n) {
        items_.push_back({(void**)slot, (size_t)std::max<int64_t>(n, 0) * sizeof(T)});
    }
    int alloc(Scratch& into, bool zero, unsigned char** block = nullptr, size_t* bytes = nullptr) {
        if (items_.empty()) return FAST_OK;
        size_t total = 0;
        for (auto& it : items_) total += piece(it.bytes);
        unsigned char* b = nullptr;
        FAST_TRY(dalloc(&b, total, into.s_));
        into.v.push_back(b);
        size_t at = 0;
        for (auto& it : items_) {
            *it.slot = b + at;
            at += piece(it.bytes);
        }
        items_.clear();
        if (block) *block = b;
        if (bytes) *bytes = total;
        if (zero) FAST_CUDA(cudaMemsetAsync(b, 0, total, into.s_));
        return FAST_OK;
    }

  private:
    static size_t piece(size_t b) { return (std::max<size_t>(b, 1) + 255) / 256 * 256; }
    struct Item {
        void** slot;
        size_t bytes;
    };
    std::vector<Item> items_;
};

// Descriptors and their item (or tile) offsets, uploaded with one copy.
template <class D>
int upload(const std::vector<D>& desc, const std::vector<int64_t>& off, Scratch& sc, const D** d_desc,
           const int64_t** d_off) {
    const size_t a = (desc.size() * sizeof(D) + 15) / 16 * 16;
    const size_t bytes = a + off.size() * sizeof(int64_t);
    unsigned char* b = nullptr;
    FAST_TRY(dalloc(&b, bytes, sc.s_));
    sc.v.push_back(b);
    std::vector<unsigned char> h(bytes, 0);
    memcpy(h.data(), desc.data(), desc.size() * sizeof(D));
    if (!off.empty()) memcpy(h.data() + a, off.data(), off.size() * sizeof(int64_t));
    FAST_CUDA(cudaMemcpyAsync(b, h.data(), bytes, cudaMemcpyHostToDevice, sc.s_));
    *d_desc = (const D*)b;
    *d_off = (const int64_t*)(b + a);
    return FAST_OK;
}

inline std::vector<int64_t> prefix(const std::vector<int64_t>& n) {
    std::vector<int64_t> off(n.size() + 1, 0);
    for (size_t i = 0; i < n.size(); i++) off[i + 1] = off[i] + n[i];
    return off;
}

// A plain batched kernel over segments of n_s items.
template <class D, class... X>
int run_items(void (*kernel)(const D*, const int64_t*, int, X...), const std::vector<D>& desc,
              const std::vector<int64_t>& n, cudaStream_t s, X... extra) {
    if (desc.empty()) return FAST_OK;
    const std::vector<int64_t> off = prefix(n);
    if (off.back() == 0) return FAST_OK;
    Scratch sc(s);
    const D* dd = nullptr;
    const int64_t* doff = nullptr;
    FAST_TRY(upload(desc, off, sc, &dd, &doff));
    kernel<<<items_grid(off.back()), 256, 0, s>>>(dd, doff, (int)desc.size(), extra...);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched CST step launch");
    return FAST_OK;
}

// A tile-split batched kernel over segments of e_s list entries, in tiles
// of `tile` entries, `per_block` tiles to a block of 256 threads (8: warp
// tiles; 1: block tiles).
template <class D>
int run_tiles(void (*kernel)(const D*, const int64_t*, int), const std::vector<D>& desc,
              const std::vector<int64_t>& entries, int tile, int per_block, cudaStream_t s) {
    if (desc.empty()) return FAST_OK;
    std::vector<int64_t> t(entries.size());
    for (size_t i = 0; i < entries.size(); i++) t[i] = ceil_div(entries[i], (int64_t)tile);
    const std::vector<int64_t> off = prefix(t);
    if (off.back() == 0) return FAST_OK;
    Scratch sc(s);
    const D* dd = nullptr;
    const int64_t* doff = nullptr;
    FAST_TRY(upload(desc, off, sc, &dd, &doff));
    const int64_t grid = std::min<int64_t>(ceil_div(off.back(), (int64_t)per_block), (int64_t)num_sms() * 8);
    kernel<<<(unsigned)grid, 256, 0, s>>>(dd, doff, (int)desc.size());
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched CST step launch");
    return FAST_OK;
}

// Size words on the device: field f of query q at Z[f * nq + q].  The
// filter counts are by query vertex, the rest by BFS position.
enum : int {
    F_CNT = 0,                    // |C0(u)|
    F_TD = F_CNT + kMaxK,         // |C_td| of the vertex at position t
    F_E = F_TD + kMaxK,           // its top-down edge space
    F_KEPT = F_E + kMaxK,         // its top-down list entries
    F_C = F_KEPT + kMaxK,         // |C| after refinement
    F_T = F_C + kMaxK,            // its tree-list entries after refinement
    F_W = F_T + kMaxK,            // W, saturating uint64
    F_WF = F_W + 1,               // W, float64
    F_END = F_WF + 1
};

// Batches of at most this many queries, whose bounded top-down arrays fit
// in kBoundedBytes, build the top-down pass without host round trips.
constexpr int kBoundedQueries = 8;
constexpr uint64_t kBoundedBytes = 2ull << 30;

// One query of the batch.
struct Q {
    int idx = 0;                  // in the caller's arrays
    fast_cst* c = nullptr;
    int k = 0;
    bool nlf = false;
    bool nt_refine = false;       // refine rule 2: the non-tree test in the bottom-up pass
    uint32_t* root_bits = nullptr; // rule 2: bitmap of C_td(root) for the test
    int A[kMaxK][kMaxK] = {};
    int dq[kMaxK] = {};
    int bpos[kMaxK] = {};         // vertex -> BFS position
    int64_t lo[kMaxK] = {}, hi[kMaxK] = {};
    int64_t c0[kMaxK] = {};       // |C0(u)|
    int64_t ctd[kMaxK] = {};      // |C_td(u)|
    int64_t E[kMaxK] = {};        // top-down edge space into u
    int64_t kept[kMaxK] = {};     // top-down entries kept into u
    int32_t* td_cand[kMaxK] = {};
    int32_t* td_list[kMaxK] = {};
    int64_t* td_off[kMaxK] = {};
    uint32_t* alive[kMaxK] = {};  // reached bitmap, then the bitmap of the refined C(u)
    uint32_t* rank[kMaxK] = {};
    uint2* packed[kMaxK] = {};    // {alive, rank} word pairs of the refined C(u)
    uint32_t* nlfb[kMaxK] = {};   // label-frequency pass bitmaps
    int64_t* e_off = nullptr;     // the current step's edge space
    int64_t* seg = nullptr;
};

// Matching order and non-tree edges of one query from its refined candidate
// counts, by the rules the per-query build uses.
void order_and_nontree(const Q& q, fast_cst* c) {
    fast::matching_order(q.k, q.A, c->root, c->parent, c->bfs, c->ncand, c->cfg.order_rule, c->order, c->pos);
    c->nnt = nontree_edges(q.k, q.A, c->order, c->parent, c->nt_from, c->nt_to);
}

thread_local uint64_t t_round_trips = 0;   // this thread's last batched build

int fetch(const int64_t* d, std::vector<int64_t>& h, size_t words, cudaStream_t s) {
    t_round_trips++;
    h.assign(words, 0);
    if (!words) return FAST_OK;
    cudaError_t e = cudaMemcpyAsync(h.data(), d, words * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? FAST_OK : cuda_status(e, "batched CST sizes", __FILE__, __LINE__);
}

// After the last round trip every size is known: every CST's arrays go
// into one exact-size block of its own arena, all CSTs with one launch.
int copy_to_arenas(std::vector<Q>& Qs, cudaStream_t s) {
    std::vector<CopyDesc> cd;
    uint64_t pieces = 0;
    for (auto& q : Qs) {
        fast_cst* c = q.c;
        struct Item { void** slot; uint64_t bytes; };
        std::vector<Item> items;
        for (int u = 0; u < c->k; u++) {
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
        uint64_t at = 0;
        for (auto& it : items) {
            unsigned char* dst = base + at;
            at += (std::max<uint64_t>(it.bytes, 1) + 255) / 256 * 256;
            if (it.bytes) {
                cd.push_back({(const unsigned char*)*it.slot, dst, it.bytes, pieces});
                pieces += (it.bytes + kPiece - 1) / kPiece;
            }
            *it.slot = dst;
        }
    }
    if (cd.empty()) return FAST_OK;
    Scratch sc(s);
    const CopyDesc* dd = nullptr;
    const int64_t* unused = nullptr;
    FAST_TRY(upload(cd, std::vector<int64_t>(), sc, &dd, &unused));
    const unsigned grid = (unsigned)std::min<uint64_t>(pieces, (uint64_t)num_sms() * 8);
    k_copy_many<<<grid, 256, 0, s>>>(dd, (int)cd.size(), pieces);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched CST copy launch");
    return FAST_OK;
}

// Builds every CST of Qs (all valid queries) on stream s.
int build_all(const fast_graph* g, std::vector<Q>& Qs, cudaStream_t s) {
    const int nq = (int)Qs.size();
    const int64_t n = g->n;
    const int64_t nw = n / 32 + 1;
    const GraphRuns G = graph_runs(g);
    int K = 0;
    for (auto& q : Qs) K = std::max(K, q.k);
    Scratch keep(s);                       // until the exact copies are made
    Scratch td(s);                         // top-down lists: until the bottom-up is done
    std::vector<int64_t> h;

    int64_t* Z = nullptr;
    {
        Carver cv;
        cv.add(&Z, (int64_t)F_END * nq);
        FAST_TRY(cv.alloc(keep, true));
    }
    auto zp = [&](int f, int qi) { return Z + (int64_t)f * nq + qi; };

    // ------------------------------------------------------------ filter
    //
    // Pairs with the same label, query degree and (label-frequency rule)
    // requirement have the same C0: one of them is filtered, the others
    // share its bitmap and take its count.
    std::vector<std::pair<int, int>> alias((size_t)kMaxK * nq, {-1, -1});   // [u * nq + qi] -> its pair
    {
        std::vector<FilterDesc> fd;
        std::vector<std::pair<int, int>> rep;             // fd[i]'s (query, vertex)
        std::map<std::vector<int64_t>, int> seen;
        Carver cv;
        int64_t maxb = 1;
        for (int qi = 0; qi < nq; qi++) {
            Q& q = Qs[qi];
            for (int u = 0; u < q.k; u++) {
                const int32_t l = q.c->qlabel[u];
                if (l < g->num_labels) { q.lo[u] = g->lab_ptr_host[l]; q.hi[u] = g->lab_ptr_host[l + 1]; }
                else { q.lo[u] = q.hi[u] = 0; }
                FilterDesc d;
                memset(&d, 0, sizeof(d));
                d.lo = q.lo[u];
                d.hi = q.hi[u];
                d.dq = q.dq[u];
                d.nlf = q.nlf ? 1 : 0;
                std::vector<int64_t> key{d.lo, d.hi, d.dq, d.nlf};
                if (q.nlf) {
                    for (int w = 0; w < q.k; w++) {
                        if (!q.A[u][w]) continue;
                        const int32_t lw = q.c->qlabel[w];
                        int t = 0;
                        while (t < d.r.nn && d.r.lab[t] != lw) t++;
                        if (t == d.r.nn) { d.r.lab[t] = lw; d.r.need[t] = 0; d.r.nn++; }
                        d.r.need[t]++;
                    }
                    // in label order, so that equal requirements give equal keys
                    for (int a = 1; a < d.r.nn; a++)
                        for (int b = a; b > 0 && d.r.lab[b - 1] > d.r.lab[b]; b--) {
                            std::swap(d.r.lab[b - 1], d.r.lab[b]);
                            std::swap(d.r.need[b - 1], d.r.need[b]);
                        }
                    for (int t = 0; t < d.r.nn; t++) { key.push_back(d.r.lab[t]); key.push_back(d.r.need[t]); }
                }
                auto it = seen.find(key);
                if (it != seen.end()) {
                    alias[(size_t)u * nq + qi] = rep[it->second];
                    continue;
                }
                seen.emplace(std::move(key), (int)fd.size());
                rep.push_back({qi, u});
                fd.push_back(d);
                maxb = std::max<int64_t>(maxb, q.hi[u] - q.lo[u]);
                if (q.nlf) cv.add(&q.nlfb[u], nw);
            }
        }
        FAST_TRY(cv.alloc(keep, true));
        for (size_t i = 0; i < fd.size(); i++) {
            const Q& q = Qs[rep[i].first];
            if (q.nlf) fd[i].bits = q.nlfb[rep[i].second];
            fd[i].cnt = (unsigned long long*)zp(F_CNT + rep[i].second, rep[i].first);
        }
        for (int qi = 0; qi < nq; qi++)
            for (int u = 0; u < Qs[qi].k; u++) {
                const auto a = alias[(size_t)u * nq + qi];
                if (a.first >= 0 && Qs[qi].nlf) Qs[qi].nlfb[u] = Qs[a.first].nlfb[a.second];
            }
        Scratch sc(s);
        const FilterDesc* dd = nullptr;
        const int64_t* unused = nullptr;
        FAST_TRY(upload(fd, std::vector<int64_t>(), sc, &dd, &unused));
        const int64_t np = (int64_t)fd.size();
        const int64_t x = std::max<int64_t>(1, std::min<int64_t>({ceil_div(maxb, 256), (int64_t)1024,
                                                                  ceil_div((int64_t)num_sms() * 32, np)}));
        k_filter_b<<<dim3((unsigned)x, (unsigned)np), 256, 0, s>>>(dd, g->lab_vtx, g->key, G, g->col, g->label);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched filter launch");
    }
    FAST_TRY(fetch(zp(F_CNT, 0), h, (size_t)kMaxK * nq, s));
    for (int qi = 0; qi < nq; qi++)
        for (int u = 0; u < Qs[qi].k; u++) {
            const auto a = alias[(size_t)u * nq + qi];
            if (a.first >= 0) h[(size_t)u * nq + qi] = h[(size_t)a.second * nq + a.first];
        }

    // ------------------------------------------------- root and t_q
    for (int qi = 0; qi < nq; qi++) {
        Q& q = Qs[qi];
        fast_cst* c = q.c;
        const int k = q.k;
        for (int u = 0; u < k; u++) q.c0[u] = h[(size_t)u * nq + qi];
        const int r = choose_root(k, q.c0, q.dq);
        c->root = r;
        bfs_tree(k, q.A, r, c->bfs, c->parent);
        for (int t = 0; t < k; t++) q.bpos[c->bfs[t]] = t;
    }

    // ------------------------------------------------ C(root) = C0(root)
    {
        Carver cv;
        for (auto& q : Qs) cv.add(&q.td_cand[q.c->root], q.c0[q.c->root]);
        FAST_TRY(cv.alloc(td, false));
        std::vector<CompactSeg<FilterF>> cs;
        for (int qi = 0; qi < nq; qi++) {
            const Q& q = Qs[qi];
            const int r = q.c->root;
            FilterF f{g->lab_vtx + q.lo[r], g->key, q.dq[r], q.nlf ? q.nlfb[r] : nullptr};
            cs.push_back({f, q.hi[r] - q.lo[r], q.td_cand[r], zp(F_TD + 0, qi)});
        }
        FAST_TRY(compact_seg(cs, s));
    }

    // ----------------------------------------------------- top-down
    //
    // A small batch enqueues the whole pass with no host round trip: each
    // level's arrays are sized by bounds the host knows -- the rows by
    // |C0(parent)|, the edge space by the graph's count of adjacency entries
    // from label l(parent) to label l(u) -- and the kernels read the real
    // sizes on the device (rows from the previous level's count, the edge
    // space's end from its offsets).  Otherwise, or when the bounds would
    // take too much memory, each level fetches its exact sizes first.
    bool bounded = false;
    if (!g->lab_pair_host.empty() && nq <= kBoundedQueries) {
        const int L = g->num_labels;
        uint64_t bytes = 0;
        for (auto& q : Qs)
            for (int t = 1; t < q.k; t++) {
                const int u = q.c->bfs[t], p = q.c->parent[u];
                const int32_t lp = q.c->qlabel[p], lu = q.c->qlabel[u];
                const int64_t e = (lp < L && lu < L) ? g->lab_pair_host[(size_t)lp * L + lu] : 0;
                bytes += 4ull * (uint64_t)e + 24ull * (uint64_t)(q.c0[p] + 1);
            }
        bounded = bytes <= kBoundedBytes;
    }
    auto rows_of = [&](const Q& q, int p) { return bounded ? q.c0[p] : q.ctd[p]; };
    std::vector<unsigned char*> alive_blk(kMaxK, nullptr);
    std::vector<size_t> alive_bytes(kMaxK, 0);
    std::vector<int> act;
    for (int t = 1; t < K; t++) {
        act.clear();
        for (int qi = 0; qi < nq; qi++) if (Qs[qi].k > t) act.push_back(qi);
        if (!bounded) {
            FAST_TRY(fetch(zp(F_TD + t - 1, 0), h, (size_t)nq, s));
            for (int qi = 0; qi < nq; qi++)
                if (Qs[qi].k > t - 1) Qs[qi].ctd[Qs[qi].c->bfs[t - 1]] = h[qi];
        }
        Scratch lvl(s);
        {
            Carver cv;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int64_t rows = rows_of(q, q.c->parent[q.c->bfs[t]]);
                cv.add(&q.e_off, rows + 1);
                cv.add(&q.seg, rows);
            }
            FAST_TRY(cv.alloc(lvl, false));
        }
        std::vector<int64_t> ni;
        {
            std::vector<CandSegDesc> cd;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t], p = q.c->parent[u];
                const int64_t rows = rows_of(q, p);
                cd.push_back({q.td_cand[p], rows, bounded ? zp(F_TD + q.bpos[p], qi) : nullptr, q.c->qlabel[u], q.seg,
                              q.e_off});
                ni.push_back(rows + 1);
            }
            FAST_TRY(run_items(k_cand_segment_b, cd, ni, s, G));
            std::vector<ScanSeg<int64_t>> sc;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int64_t rows = rows_of(q, q.c->parent[q.c->bfs[t]]);
                sc.push_back({q.e_off, nullptr, q.e_off, rows + 1, zp(F_E + t, qi)});
            }
            FAST_TRY(scan_seg(sc, s));
        }
        if (!bounded) FAST_TRY(fetch(zp(F_E + t, 0), h, (size_t)nq, s));
        {
            Carver cl, cb;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t], p = q.c->parent[u];
                const int64_t rows = rows_of(q, p);
                const int L = g->num_labels;
                const int32_t lp = q.c->qlabel[p], lu = q.c->qlabel[u];
                q.E[u] = !bounded ? h[qi] : (lp < L && lu < L) ? g->lab_pair_host[(size_t)lp * L + lu] : 0;
                cl.add(&q.td_list[u], q.E[u]);
                cl.add(&q.td_off[u], rows + 1);
                cb.add(&q.alive[u], nw);
            }
            FAST_TRY(cl.alloc(td, false));
            FAST_TRY(cb.alloc(keep, true, &alive_blk[t], &alive_bytes[t]));
        }
        {
            std::vector<CompactSeg<TopDownF>> cs;
            std::vector<FillTailDesc> ft;
            ni.clear();
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                const int64_t rows = rows_of(q, q.c->parent[u]);
                TopDownF f{};
                f.e_off = q.e_off; f.rows = rows; f.seg = q.seg; f.col = g->col; f.key = g->key;
                f.want_key_hi = q.c->qlabel[u]; f.want_dq = q.dq[u]; f.reached = q.alive[u]; f.t_off = q.td_off[u];
                f.label_known = G.run_ptr != nullptr;
                f.pass = q.nlf ? q.nlfb[u] : nullptr;
                f.E = q.e_off + rows;
                cs.push_back({f, q.E[u], q.td_list[u], zp(F_KEPT + t, qi)});
                ft.push_back({q.e_off, rows, zp(F_KEPT + t, qi), q.td_off[u]});
                ni.push_back(rows + 1);
            }
            FAST_TRY(compact_seg(cs, s));
            FAST_TRY(run_items(k_fill_tail_b, ft, ni, s));
        }
        {
            Carver cv;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                cv.add(&q.td_cand[u], q.c0[u]);      // C_td(u) lies inside C0(u)
            }
            FAST_TRY(cv.alloc(td, false));
            std::vector<BitsSeg> bs;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                bs.push_back({q.alive[u], n, q.td_cand[u], zp(F_TD + t, qi)});
            }
            FAST_TRY(bits_ids_seg(bs, s));
        }
    }
    // |C_td|, edge spaces and kept entries of every position
    FAST_TRY(fetch(zp(F_TD, 0), h, (size_t)3 * kMaxK * nq, s));
    for (int qi = 0; qi < nq; qi++) {
        Q& q = Qs[qi];
        for (int t = 0; t < q.k; t++) {
            const int u = q.c->bfs[t];
            q.ctd[u] = h[(size_t)t * nq + qi];
            q.kept[u] = h[(size_t)(2 * kMaxK + t) * nq + qi];
            // a bounded pass read at most its bound of each edge space (the
            // compaction stops there); more would mean a wrong bound
            if (bounded && t > 0 && h[(size_t)(kMaxK + t) * nq + qi] > q.E[u])
                return set_error(FAST_ERR_CUDA, "batched CST build: an edge space exceeded its label-pair bound");
        }
    }

    // refine rule 2 tests against C_td(root) until the root's own step: its
    // bitmap (the other vertices' top-down bitmaps already exist)
    {
        Carver cv;
        std::vector<SetBitsDesc> sb;
        std::vector<int64_t> ni;
        for (auto& q : Qs)
            if (q.nt_refine) cv.add(&q.root_bits, nw);
        FAST_TRY(cv.alloc(keep, true));
        for (int qi = 0; qi < nq; qi++) {
            Q& q = Qs[qi];
            if (!q.nt_refine) continue;
            const int r = q.c->root;
            sb.push_back({q.td_cand[r], zp(F_TD + 0, qi), q.root_bits});
            ni.push_back(q.ctd[r]);
        }
        FAST_TRY(run_items(k_set_bits_b, sb, ni, s));
    }

    // ---------------------------------------------------- bottom-up
    for (int t = K - 1; t >= 0; t--) {
        act.clear();
        for (int qi = 0; qi < nq; qi++) if (Qs[qi].k > t) act.push_back(qi);
        Scratch lvl(s);
        // (query, child) pairs, grouped by query in act order
        std::vector<int> pa, pw, pbeg(act.size() + 1, 0);
        for (size_t a = 0; a < act.size(); a++) {
            const Q& q = Qs[act[a]];
            const int u = q.c->bfs[t];
            for (int w = 0; w < q.k; w++)
                if (q.c->parent[w] == u) { pa.push_back((int)a); pw.push_back(w); }
            pbeg[a + 1] = (int)pa.size();
        }
        const size_t npr = pa.size();
        std::vector<uint8_t*> has(npr, nullptr);
        std::vector<uint8_t*> valid(act.size(), nullptr);
        std::vector<int64_t*> newrow(act.size(), nullptr);
        {
            Carver ch, cv;
            for (size_t j = 0; j < npr; j++) {
                const Q& q = Qs[act[pa[j]]];
                ch.add(&has[j], q.ctd[q.c->bfs[t]]);
            }
            for (size_t a = 0; a < act.size(); a++) {
                const Q& q = Qs[act[a]];
                const int64_t rows = q.ctd[q.c->bfs[t]];
                cv.add(&valid[a], rows);
                cv.add(&newrow[a], rows + 1);
            }
            FAST_TRY(ch.alloc(lvl, true));
            FAST_TRY(cv.alloc(lvl, false));
        }
        {
            std::vector<AnyAliveDesc> aa;
            std::vector<int64_t> ent;
            for (size_t j = 0; j < npr; j++) {
                const Q& q = Qs[act[pa[j]]];
                const int w = pw[j];
                aa.push_back({q.td_off[w], q.ctd[q.c->bfs[t]], q.td_list[w], q.alive[w], has[j]});
                ent.push_back(q.kept[w]);
            }
            FAST_TRY(run_tiles(k_any_alive_b, aa, ent, kTileItems, 1, s));
        }
        // refine rule 2: per (query, non-tree neighbour w of u), which rows
        // have a neighbour in C(w) as it stands now
        std::vector<int> na, nwv, nbeg(act.size() + 1, 0);
        for (size_t a = 0; a < act.size(); a++) {
            const Q& q = Qs[act[a]];
            const int u = q.c->bfs[t];
            if (q.nt_refine)
                for (int w = 0; w < q.k; w++)
                    if (q.A[u][w] && q.c->parent[w] != u && q.c->parent[u] != w) { na.push_back((int)a); nwv.push_back(w); }
            nbeg[a + 1] = (int)na.size();
        }
        std::vector<uint8_t*> ntf(na.size(), nullptr);
        if (!na.empty()) {
            Carver cf;
            for (size_t j = 0; j < na.size(); j++) {
                const Q& q = Qs[act[na[j]]];
                cf.add(&ntf[j], q.ctd[q.c->bfs[t]]);
            }
            FAST_TRY(cf.alloc(lvl, true));
            std::vector<NtDesc> nd;
            std::vector<int64_t> ni;
            for (size_t j = 0; j < na.size(); j++) {
                const Q& q = Qs[act[na[j]]];
                const int u = q.c->bfs[t], w = nwv[j];
                // later in the BFS order: already refined; earlier: its
                // top-down set (the root's own bitmap; the others' reached
                // bitmaps are not rewritten before their step)
                const uint32_t* bits = (w == q.c->root && q.bpos[w] < t) ? q.root_bits : q.alive[w];
                nd.push_back({q.td_cand[u], q.c->qlabel[w], bits, ntf[j]});
                ni.push_back(q.ctd[u]);
            }
            if (!nd.empty()) {
                const std::vector<int64_t> off = prefix(ni);
                if (off.back() > 0) {
                    Scratch sc(s);
                    const NtDesc* dd = nullptr;
                    const int64_t* doff = nullptr;
                    FAST_TRY(upload(nd, off, sc, &dd, &doff));
                    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(off.back(), 8),
                                                                                  (int64_t)num_sms() * 16));
                    k_nt_support_b<<<(unsigned)blocks, 256, 0, s>>>(dd, doff, (int)nd.size(), G, g->col);
                    note_launch();
                    if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched non-tree test launch");
                }
            }
        }
        {
            std::vector<ValidDesc> vd;
            std::vector<int64_t> ni;
            std::vector<ScanSeg<int64_t>> sc;
            for (size_t a = 0; a < act.size(); a++) {
                const Q& q = Qs[act[a]];
                const int64_t rows = q.ctd[q.c->bfs[t]];
                ValidDesc d;
                memset(&d, 0, sizeof(d));
                for (int j = pbeg[a]; j < pbeg[a + 1]; j++) d.cf.has[d.cf.nch++] = has[j];
                for (int j = nbeg[a]; j < nbeg[a + 1]; j++) d.cf.has[d.cf.nch++] = ntf[j];
                d.valid = valid[a];
                d.vflag = newrow[a];
                vd.push_back(d);
                ni.push_back(rows);
                sc.push_back({newrow[a], nullptr, newrow[a], rows, newrow[a] + rows});
            }
            FAST_TRY(run_items(k_valid_rows_b, vd, ni, s));
            FAST_TRY(scan_seg(sc, s));
        }
        {
            Carver cv;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                cv.add(&q.c->cand[u], q.ctd[u]);
            }
            for (size_t j = 0; j < npr; j++) {
                Q& q = Qs[act[pa[j]]];
                const int w = pw[j];
                cv.add(&q.c->t_off[w], q.ctd[q.c->bfs[t]] + 1);
                cv.add(&q.c->t_idx[w], q.kept[w]);
            }
            FAST_TRY(cv.alloc(keep, false));
            std::vector<CompactSeg<KeepRowsF>> kr;
            for (size_t a = 0; a < act.size(); a++) {
                const int qi = act[a];
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                kr.push_back({KeepRowsF{q.td_cand[u], valid[a], zp(F_TD + t, qi)}, q.ctd[u], q.c->cand[u], zp(F_C + t, qi)});
            }
            FAST_TRY(compact_seg(kr, s));
            std::vector<CompactSeg<WriteAliveF>> wa;
            std::vector<SetTailDesc> st;
            for (size_t j = 0; j < npr; j++) {
                const int a = pa[j], qi = act[a];
                Q& q = Qs[qi];
                const int w = pw[j];
                WriteAliveF f{};
                f.off = q.td_off[w]; f.nrows = zp(F_TD + t, qi); f.list = q.td_list[w];
                f.alive = q.alive[w]; f.rank = q.rank[w]; f.packed = q.packed[w];
                f.valid = valid[a]; f.newrow = newrow[a]; f.new_off = q.c->t_off[w];
                wa.push_back({f, q.kept[w], q.c->t_idx[w], zp(F_T + q.bpos[w], qi)});
                st.push_back({q.c->t_off[w], zp(F_C + t, qi), zp(F_T + q.bpos[w], qi)});
            }
            FAST_TRY(compact_seg(wa, s));
            if (!st.empty()) {
                Scratch sc(s);
                const SetTailDesc* dd = nullptr;
                const int64_t* unused = nullptr;
                FAST_TRY(upload(st, std::vector<int64_t>(), sc, &dd, &unused));
                k_set_tail_b<<<(unsigned)ceil_div((int64_t)st.size(), 256), 256, 0, s>>>(dd, (int)st.size());
                note_launch();
                if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched set-tail launch");
            }
        }
        // bitmap and rank of the refined C(u)
        if (t == 0) {
            Carver cv;
            for (int qi : act) cv.add(&Qs[qi].alive[Qs[qi].c->root], nw);
            FAST_TRY(cv.alloc(keep, true));
        } else {
            FAST_CUDA(cudaMemsetAsync(alive_blk[t], 0, alive_bytes[t], s));
        }
        {
            std::vector<SetBitsDesc> sb;
            std::vector<int64_t> ni;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                sb.push_back({q.c->cand[u], zp(F_C + t, qi), q.alive[u]});
                ni.push_back(q.ctd[u]);
            }
            FAST_TRY(run_items(k_set_bits_b, sb, ni, s));
            Carver cv;
            for (int qi : act) cv.add(&Qs[qi].rank[Qs[qi].c->bfs[t]], nw);
            FAST_TRY(cv.alloc(keep, false));
            std::vector<ScanSeg<uint32_t>> rk;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                rk.push_back({nullptr, q.alive[u], q.rank[u], nw, nullptr});
            }
            FAST_TRY(scan_seg(rk, s));
            Carver cp;
            for (int qi : act) cp.add(&Qs[qi].packed[Qs[qi].c->bfs[t]], nw);
            FAST_TRY(cp.alloc(keep, false));
            std::vector<PackDesc> pd;
            std::vector<int64_t> pn;
            for (int qi : act) {
                Q& q = Qs[qi];
                const int u = q.c->bfs[t];
                pd.push_back({q.alive[u], q.rank[u], q.packed[u]});
                pn.push_back(nw);
            }
            FAST_TRY(run_items(k_pack_bits_b, pd, pn, s));
        }
    }
    td.release();                          // top-down lists and sets: done
    // refined candidate counts decide the matching order
    FAST_TRY(fetch(zp(F_C, 0), h, (size_t)2 * kMaxK * nq, s));
    for (int qi = 0; qi < nq; qi++) {
        Q& q = Qs[qi];
        fast_cst* c = q.c;
        for (int t = 0; t < q.k; t++) {
            const int u = c->bfs[t];
            c->ncand[u] = h[(size_t)t * nq + qi];
            c->t_entries[u] = c->parent[u] < 0 ? 0 : h[(size_t)(kMaxK + t) * nq + qi];
        }
        order_and_nontree(q, c);
    }

    // ------------------------------------------------------ non-tree
    std::vector<int> ntq, nte;                       // (query, edge) pairs
    for (int qi = 0; qi < nq; qi++)
        for (int e = 0; e < Qs[qi].c->nnt; e++) { ntq.push_back(qi); nte.push_back(e); }
    const size_t nnp = ntq.size();
    int64_t* NZ = nullptr;                           // [0, nnp) edge spaces, [nnp, 2 nnp) kept entries
    if (nnp) {
        Carver cz;
        cz.add(&NZ, (int64_t)(2 * nnp));
        FAST_TRY(cz.alloc(keep, true));
        Scratch lvl(s);
        std::vector<int64_t*> eo(nnp, nullptr), sg(nnp, nullptr);
        std::vector<int64_t> rows(nnp);
        {
            Carver cv;
            for (size_t j = 0; j < nnp; j++) {
                const fast_cst* c = Qs[ntq[j]].c;
                rows[j] = c->ncand[c->nt_from[nte[j]]];
                cv.add(&eo[j], rows[j] + 1);
                cv.add(&sg[j], rows[j]);
            }
            FAST_TRY(cv.alloc(lvl, false));
        }
        {
            std::vector<CandSegDesc> cd;
            std::vector<int64_t> ni;
            std::vector<ScanSeg<int64_t>> sc;
            for (size_t j = 0; j < nnp; j++) {
                const fast_cst* c = Qs[ntq[j]].c;
                const int e = nte[j];
                cd.push_back({c->cand[c->nt_from[e]], rows[j], nullptr, c->qlabel[c->nt_to[e]], sg[j], eo[j]});
                ni.push_back(rows[j] + 1);
                sc.push_back({eo[j], nullptr, eo[j], rows[j] + 1, NZ + j});
            }
            FAST_TRY(run_items(k_cand_segment_b, cd, ni, s, G));
            FAST_TRY(scan_seg(sc, s));
        }
        FAST_TRY(fetch(NZ, h, nnp, s));
        {
            Carver cv;
            for (size_t j = 0; j < nnp; j++) {
                fast_cst* c = Qs[ntq[j]].c;
                const int e = nte[j];
                cv.add(&c->n_off[e], rows[j] + 1);
                cv.add(&c->n_idx[e], h[j]);
            }
            FAST_TRY(cv.alloc(keep, false));
            std::vector<CompactSeg<NonTreeF>> cs;
            std::vector<FillTailDesc> ft;
            std::vector<int64_t> ni;
            for (size_t j = 0; j < nnp; j++) {
                const Q& q = Qs[ntq[j]];
                fast_cst* c = q.c;
                const int e = nte[j], ui = c->nt_to[e];
                NonTreeF f{};
                f.e_off = eo[j]; f.rows = rows[j]; f.seg = sg[j]; f.col = g->col;
                f.alive = q.alive[ui]; f.rank = q.rank[ui]; f.packed = q.packed[ui]; f.n_off = c->n_off[e];
                f.E = eo[j] + rows[j];
                cs.push_back({f, h[j], c->n_idx[e], NZ + nnp + j});
                ft.push_back({eo[j], rows[j], NZ + nnp + j, c->n_off[e]});
                ni.push_back(rows[j] + 1);
            }
            FAST_TRY(compact_seg(cs, s));
            FAST_TRY(run_items(k_fill_tail_b, ft, ni, s));
        }
    }

    // ------------------------------------------------------ workload
    for (int t = K - 1; t >= 0; t--) {
        act.clear();
        for (int qi = 0; qi < nq; qi++) if (Qs[qi].k > t) act.push_back(qi);
        std::vector<int> pa, pw, pbeg(act.size() + 1, 0);
        for (size_t a = 0; a < act.size(); a++) {
            const Q& q = Qs[act[a]];
            const int u = q.c->bfs[t];
            for (int w = 0; w < q.k; w++)
                if (q.c->parent[w] == u) { pa.push_back((int)a); pw.push_back(w); }
            pbeg[a + 1] = (int)pa.size();
        }
        const size_t npr = pa.size();
        std::vector<double*> sumf(npr, nullptr);
        std::vector<uint32_t*> ovf(npr, nullptr);
        {
            Carver cv, cz;
            for (int qi : act) {
                fast_cst* c = Qs[qi].c;
                const int u = c->bfs[t];
                cv.add(&c->cval[u], c->ncand[u]);
                cv.add(&c->cvalf[u], c->ncand[u]);
            }
            for (size_t j = 0; j < npr; j++) {
                fast_cst* c = Qs[act[pa[j]]].c;
                const int64_t rows = c->ncand[c->bfs[t]];
                cz.add(&c->ssum[pw[j]], rows);
                cz.add(&sumf[j], rows);
                cz.add(&ovf[j], rows);
            }
            FAST_TRY(cv.alloc(keep, false));
            FAST_TRY(cz.alloc(keep, true));
        }
        {
            std::vector<ChildSumDesc> cd;
            std::vector<int64_t> ent;
            for (size_t j = 0; j < npr; j++) {
                fast_cst* c = Qs[act[pa[j]]].c;
                const int w = pw[j];
                cd.push_back({c->t_off[w], c->ncand[c->bfs[t]], c->t_idx[w], c->cval[w], c->cvalf[w],
                              (unsigned long long*)c->ssum[w], sumf[j], ovf[j]});
                ent.push_back(c->t_entries[w]);
            }
            FAST_TRY(run_tiles(k_child_sums_b, cd, ent, kWarpTileItems, 8, s));
        }
        {
            std::vector<ProdDesc> pd;
            std::vector<int64_t> ni;
            for (size_t a = 0; a < act.size(); a++) {
                fast_cst* c = Qs[act[a]].c;
                const int u = c->bfs[t];
                ProdDesc d;
                memset(&d, 0, sizeof(d));
                for (int j = pbeg[a]; j < pbeg[a + 1]; j++) {
                    const int i = d.cs.nch++;
                    d.cs.ssum[i] = c->ssum[pw[j]];
                    d.cs.sumf[i] = sumf[j];
                    d.cs.ovf[i] = ovf[j];
                }
                d.cval = c->cval[u];
                d.cvalf = c->cvalf[u];
                pd.push_back(d);
                ni.push_back(c->ncand[u]);
            }
            FAST_TRY(run_items(k_workload_prod_b, pd, ni, s));
        }
    }
    {
        std::vector<TotalDesc> td_;
        for (int qi = 0; qi < nq; qi++) {
            fast_cst* c = Qs[qi].c;
            td_.push_back({c->cval[c->root], c->cvalf[c->root], c->ncand[c->root], (uint64_t*)zp(F_W, qi),
                           (double*)zp(F_WF, qi)});
        }
        Scratch sc(s);
        const TotalDesc* dd = nullptr;
        const int64_t* unused = nullptr;
        FAST_TRY(upload(td_, std::vector<int64_t>(), sc, &dd, &unused));
        k_total_w_b<<<(unsigned)nq, 1024, 0, s>>>(dd);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) return set_error(FAST_ERR_CUDA, "batched W launch");
    }

    // ---------------------------------------- the last round trip
    {
        std::vector<int64_t> hw, hk;
        FAST_TRY(fetch(zp(F_W, 0), hw, (size_t)2 * nq, s));
        if (nnp) FAST_TRY(fetch(NZ + nnp, hk, nnp, s));
        int lb_err = 0;
        cudaError_t e = cudaMemcpyFromSymbolAsync(&lb_err, g_lookback_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e, "batched CST build", __FILE__, __LINE__);
        if (lb_err) return set_error(FAST_ERR_CUDA, "batched CST build: a look-back wait ran out");
        for (int qi = 0; qi < nq; qi++) {
            memcpy(&Qs[qi].c->W, &hw[qi], sizeof(uint64_t));
            memcpy(&Qs[qi].c->Wf, &hw[(size_t)nq + qi], sizeof(double));
        }
        for (size_t j = 0; j < nnp; j++) Qs[ntq[j]].c->n_entries[nte[j]] = hk[j];
    }
    return copy_to_arenas(Qs, s);
}

// Queries per group: bounds the grid's y extent of the filter launch
// (queries x vertices <= 65535) and the scratch held at once.
constexpr int kGroup = 1024;

}  // namespace

namespace fast {

int build_cst_batch(const fast_graph* g, int32_t nq, const fast_query_desc* qs, const fast_config* const* cfgs,
                    cudaStream_t s, fast_cst** outs, int32_t* status) {
    t_round_trips = 0;
    for (int i = 0; i < nq; i++) outs[i] = nullptr;
    // Ranges of queries built together: groups of kGroup; a range whose
    // build runs out of device memory (its bound-sized buffers did not fit)
    // is released and built as two halves, down to single queries.  The
    // CSTs do not depend on how the queries are grouped.
    std::vector<std::pair<int, int>> todo;
    for (int g0 = nq - (nq % kGroup == 0 ? kGroup : nq % kGroup); g0 >= 0; g0 -= kGroup)
        todo.push_back({g0, std::min(nq, g0 + kGroup)});
    while (!todo.empty()) {
        const int g0 = todo.back().first, g1 = todo.back().second;
        todo.pop_back();
        std::vector<Q> Qs;
        Qs.reserve(g1 - g0);
        for (int i = g0; i < g1; i++) {
            Q q;
            int rc = validate_query(&qs[i], q.A, q.dq);
            const fast_config* cf = cfgs[i];
            if (rc == FAST_OK && cf && (cf->order_rule < 0 || cf->order_rule > 3))
                rc = set_error(FAST_ERR_INVALID,
                               "fast_build_cst_batch: order_rule %d (0 path-based, 1 greedy, 2 BFS, 3 fewest candidates)",
                               cf->order_rule);
            if (rc == FAST_OK && cf && (cf->filter_rule < 0 || cf->filter_rule > 1))
                rc = set_error(FAST_ERR_INVALID,
                               "fast_build_cst_batch: filter_rule %d (0 label and degree, 1 label frequencies)",
                               cf->filter_rule);
            if (rc == FAST_OK && cf && cf->refine_rule != 0 && cf->refine_rule != 2)
                rc = set_error(FAST_ERR_INVALID, "fast_build_cst_batch: refine_rule %d (0 or 2)", cf->refine_rule);
            status[i] = rc;
            if (rc != FAST_OK) continue;
            fast_cst* c = new fast_cst();
            memset(c->cand, 0, sizeof(c->cand)); memset(c->t_off, 0, sizeof(c->t_off)); memset(c->t_idx, 0, sizeof(c->t_idx));
            memset(c->cval, 0, sizeof(c->cval)); memset(c->cvalf, 0, sizeof(c->cvalf)); memset(c->ssum, 0, sizeof(c->ssum));
            memset(c->n_off, 0, sizeof(c->n_off)); memset(c->n_idx, 0, sizeof(c->n_idx));
            memset(c->t_entries, 0, sizeof(c->t_entries)); memset(c->ncand, 0, sizeof(c->ncand));
            memset(c->n_entries, 0, sizeof(c->n_entries));
            c->g = g;
            c->k = qs[i].n;
            c->stream = s;
            if (cf) c->cfg = *cf; else fast_config_default(&c->cfg);
            for (int u = 0; u < c->k; u++) { c->qlabel[u] = qs[i].labels[u]; c->dq[u] = q.dq[u]; }
            q.idx = i;
            q.c = c;
            q.k = c->k;
            q.nlf = c->cfg.filter_rule == 1;
            q.nt_refine = c->cfg.refine_rule == 2;
            Qs.push_back(q);
        }
        int rc = Qs.empty() ? FAST_OK : build_all(g, Qs, s);
        if (rc == FAST_ERR_OOM && Qs.size() > 1) {
            for (auto& q : Qs) cst_release_nosync(q.c);
            cudaStreamSynchronize(s);              // the freed buffers are reusable by the halves
            pool_release_unused(pool_active());    // and the scratch the attempt grew goes back
            trim_freed_memory();
            set_error(FAST_OK, "%s", "");
            const int mid = g0 + (g1 - g0) / 2;
            todo.push_back({mid, g1});
            todo.push_back({g0, mid});
            continue;
        }
        if (rc != FAST_OK) {
            for (auto& q : Qs) cst_release_nosync(q.c);
            for (int i = 0; i < nq; i++) { cst_release_nosync(outs[i]); outs[i] = nullptr; }
            return rc;
        }
        for (auto& q : Qs) outs[q.idx] = q.c;
    }
    return FAST_OK;
}

}  // namespace fast

extern "C" uint64_t fast_last_build_round_trips(void) { return t_round_trips; }

extern "C" int fast_build_cst_batch(const fast_graph* g, int32_t nq, const fast_query_desc* qs, const fast_config* cfg,
                                    void* stream, fast_cst** outs, int32_t* status) {
    if (!g || nq < 0 || (nq > 0 && (!qs || !outs || !status)))
        return set_error(FAST_ERR_INVALID, "fast_build_cst_batch: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    PoolScope scratch(s);
    std::vector<const fast_config*> cfgs(nq, cfg);
    return build_cst_batch(g, nq, qs, cfgs.data(), s, outs, status);
}
