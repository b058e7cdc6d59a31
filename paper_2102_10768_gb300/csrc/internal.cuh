// Definitions of the library's opaque handles (device-resident data graph,
// candidate search tree and partition) and of the chunk descriptor shared by
// the partitioner and the matcher.
#pragma once

#include <vector>

#include "common.cuh"

constexpr int kMaxK = FAST_MAX_QUERY;
constexpr int kMaxNT = kMaxK * (kMaxK - 1) / 2;

// Data graph G (Sec. II-A) on the device.
constexpr int kLabelPairMax = 1024;

struct fast_graph {
    int64_t n = 0;
    int64_t nadj = 0;          // stored adjacency entries (2|E|)
    int32_t num_labels = 0;
    int64_t max_degree = 0;
    int64_t* row_ptr = nullptr;   // [n+1]
    int32_t* col = nullptr;       // [nadj], each row sorted ascending
    int32_t* label = nullptr;     // [n]
    int32_t* key = nullptr;       // [n] (label << 8) | min(degree, 255): one load per filter test
    int64_t* lab_ptr = nullptr;   // [num_labels+1]
    int32_t* lab_vtx = nullptr;   // [n] vertices grouped by label, ascending id
    std::vector<int64_t> lab_ptr_host;
    std::vector<int64_t> lab_degsum_host;   // per label: sum of degrees (bounds CST list sizes)
    // adjacency entries per (label of the row's vertex a, label of the
    // neighbour b) at [a * num_labels + b], when the rows are grouped by label
    // and num_labels <= kLabelPairMax (else empty): bounds a top-down list
    std::vector<int64_t> lab_pair_host;
    // Label runs: when `grouped`, each row of col is sorted by (label of the
    // neighbour, id), and row v's runs are run_ptr[v] .. run_ptr[v+1]-1: run
    // r holds the neighbours with label run_lab[r], from col position
    // run_beg[r] to the next run's start (or the row's end).
    bool grouped = false;
    int64_t* run_ptr = nullptr;   // [n+1]
    int32_t* run_lab = nullptr;   // [R]
    int64_t* run_beg = nullptr;   // [R]
};

// The neighbours of v with label l: col[*beg .. *beg + *len), ascending id.
// An ungrouped graph gives the whole row (the caller still tests labels).
struct GraphRuns {
    const int64_t* row_ptr;
    const int64_t* run_ptr;       // null: ungrouped
    const int32_t* run_lab;
    const int64_t* run_beg;
};

__device__ __forceinline__ void label_segment(const GraphRuns& G, int32_t v, int32_t l, int64_t* beg, int64_t* len) {
    const int64_t a = G.row_ptr[v], b = G.row_ptr[v + 1];
    if (!G.run_ptr) { *beg = a; *len = b - a; return; }
    int64_t lo = G.run_ptr[v], hi = G.run_ptr[v + 1];
    const int64_t r1 = hi;
    while (lo < hi) {                              // first run with label >= l
        int64_t mid = (lo + hi) >> 1;
        if (G.run_lab[mid] < l) lo = mid + 1; else hi = mid;
    }
    if (lo < r1 && G.run_lab[lo] == l) {
        *beg = G.run_beg[lo];
        *len = (lo + 1 < r1 ? G.run_beg[lo + 1] : b) - *beg;
    } else {
        *beg = a;
        *len = 0;
    }
}

inline GraphRuns graph_runs(const fast_graph* g) {
    GraphRuns G;
    G.row_ptr = g->row_ptr;
    G.run_ptr = g->grouped ? g->run_ptr : nullptr;
    G.run_lab = g->run_lab;
    G.run_beg = g->run_beg;
    return G;
}

// Candidate search tree (Sec. IV-A) of one query.  Indexed by query vertex
// unless noted; lists hold candidate-local indices.
struct fast_cst {
    const fast_graph* g = nullptr;
    int k = 0;
    int root = 0;
    int order[kMaxK];          // position -> query vertex (matching order O)
    int pos[kMaxK];            // query vertex -> position
    int parent[kMaxK];         // query vertex -> parent in t_q (-1: root)
    int bfs[kMaxK];            // BFS order of t_q
    int32_t qlabel[kMaxK];
    int32_t dq[kMaxK];         // query degree
    int64_t ncand[kMaxK];      // |C(u)|
    int32_t* cand[kMaxK];      // C(u): sorted data-vertex ids
    int64_t* t_off[kMaxK];     // tree lists into u: offsets over rows of C(parent(u))
    uint32_t* t_idx[kMaxK];    //   entries: indices into C(u)
    int64_t t_entries[kMaxK];
    int nnt = 0;
    int nt_from[kMaxNT], nt_to[kMaxNT];   // query vertices, earlier -> later in O
    int64_t* n_off[kMaxNT];
    uint32_t* n_idx[kMaxNT];
    int64_t n_entries[kMaxNT];
    uint64_t* cval[kMaxK];     // c_u(v), saturating uint64 (Sec. IV-C)
    double* cvalf[kMaxK];      // c_u(v), float64
    uint64_t* ssum[kMaxK];     // per row of C(parent(u)): sum of c_u over its list into u
    uint64_t W = 0;
    double Wf = 0.0;
    fast_config cfg;
    cudaStream_t stream = nullptr;
    fast::Arena arena;         // every array above lives in it (exact sizes)
    std::vector<void*> build_tmp;   // during fast_build_cst: bounded buffers replaced by exact copies
};

// One chunk of a partitioned CST (Sec. IV-B): positions 0..j-1 fixed to one
// candidate each (prefix, candidate-local indices), position j restricted to
// entries [a, b) of its list L_j.
struct alignas(16) Chunk {
    int32_t j;
    uint32_t a, b;
    uint32_t pad;
    uint64_t w;                // workload estimate W' (saturating)
    uint64_t id;               // sampling id
    uint32_t prefix[kMaxK];
};

struct fast_chunks {
    const fast_cst* c = nullptr;
    int64_t n = 0;
    Chunk* d = nullptr;        // device [n]
    cudaStream_t stream = nullptr;
};

namespace fast {
// Stream-ordered release without the synchronisation of the public free
// calls, for callers whose streams are already idle or stay ordered.
void cst_release_nosync(fast_cst* c);
void chunks_release_nosync(fast_chunks* ch);

// The CSTs of nq queries built together (cst_batch.cu), query i with
// cfgs[i] (NULL: defaults); outs[i] and status[i] as fast_build_cst_batch.
int build_cst_batch(const fast_graph* g, int32_t nq, const fast_query_desc* qs, const fast_config* const* cfgs,
                    cudaStream_t s, fast_cst** outs, int32_t* status);

// The partitions of nq CSTs built together (partition_batch.cu), CST i with
// cfgs[i] (NULL: its own configuration); outs[i] and status[i] as
// fast_partition_batch.
int partition_batch(const fast_cst* const* csts, int32_t nq, const fast_config* const* cfgs, cudaStream_t s,
                    fast_chunks** outs, int32_t* status);
}  // namespace fast
