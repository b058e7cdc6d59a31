// Data-graph loader (Sec. II-A data model) and the library's error plumbing.
//
// fast_load_graph turns an edge list into a device CSR of the simple
// undirected graph: both directions of every edge become 64-bit keys
// (src << 32 | dst), a stable LSD radix sort orders them, an ordered
// compaction drops self loops and repeats, and a boundary pass writes the row
// offsets.  When ids and labels fit one 64-bit key, the adjacency entries are
// re-sorted stably on (row, label of the neighbour), so that each row holds
// its neighbours grouped by label (ascending id within a label), and a
// per-row directory of label runs is built for the CST build.  A radix sort
// on (label << 32 | id) builds the label index.
#include <stdarg.h>

#include <atomic>
#include <cstring>

#include "internal.cuh"
#include "prims.cuh"

namespace fast {

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_status(cudaError_t e, const char* what, const char* file, int line) {
    cudaGetLastError();
    int code = (e == cudaErrorMemoryAllocation) ? FAST_ERR_OOM : FAST_ERR_CUDA;
    const char* base = strrchr(file, '/');
    return set_error(code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
}

}  // namespace fast

using namespace fast;

extern "C" const char* fast_last_error(void) { return g_err; }

extern "C" uint64_t fast_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" void fast_config_default(fast_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->delta_w = 1ull << 20;
    cfg->sample_root = 0.0;
    cfg->sample_deep = 0.0;
    cfg->sample_seed = 0;
    cfg->max_chunks = 1ll << 16;
    cfg->warps_per_block = 8;
    cfg->blocks_per_sm = 4;
    cfg->time_budget_s = 0.0;
    cfg->limit = 0;
    cfg->queue_cells = 0;
    cfg->order_rule = 0;
    cfg->filter_rule = 0;
    cfg->build_rule = 0;
    cfg->refine_rule = 0;
    cfg->matcher_rule = 0;
    cfg->validators = 0;
}

namespace {


__global__ void k_edge_keys(const int32_t* __restrict__ edges, int64_t m, int64_t n, uint64_t sent,
                            uint64_t* __restrict__ keys, int* __restrict__ bad) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n || b >= n) {
        atomicOr(bad, 1);
        keys[2 * e] = keys[2 * e + 1] = sent;
        return;
    }
    if (a == b) {
        keys[2 * e] = keys[2 * e + 1] = sent;
        return;
    }
    keys[2 * e] = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
    keys[2 * e + 1] = ((uint64_t)(uint32_t)b << 32) | (uint32_t)a;
}

__global__ void k_check_labels(const int32_t* __restrict__ lab, int64_t n, int* __restrict__ bad,
                               int* __restrict__ maxlab) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int32_t l = lab[v];
    if (l < 0 || l >= (1 << 23)) atomicOr(bad, 2);
    else atomicMax(maxlab, l);
}

// keep key i iff it is a real edge and differs from its predecessor
struct DedupF {
    using value_type = uint64_t;
    const uint64_t* keys;
    uint64_t sent;
    __device__ void begin(int64_t) {}
    __device__ bool eval(int64_t i, uint64_t& v) const {
        uint64_t k = keys[i];
        v = k;
        return k != sent && (i == 0 || keys[i - 1] != k);
    }
    __device__ int64_t tag(int64_t) const { return -1; }
    __device__ void at(int64_t, int64_t) const {}
};

// row_ptr[v] = first position whose source is >= v, from sorted keys
__global__ void k_row_bounds(const uint64_t* __restrict__ kept, int64_t nadj, int64_t n,
                             int64_t* __restrict__ row_ptr, int32_t* __restrict__ col) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > nadj) return;
    int64_t hi = (p < nadj) ? (int64_t)(kept[p] >> 32) : n;      // rows (prev, hi] start at p
    int64_t lo = (p == 0) ? -1 : (int64_t)(kept[p - 1] >> 32);
    for (int64_t v = lo + 1; v <= hi; v++) row_ptr[v] = p;
    if (p < nadj) col[p] = (int32_t)(kept[p] & 0xFFFFFFFFu);
}

__global__ void k_vertex_keys(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ lab, int64_t n,
                              int32_t* __restrict__ key, uint64_t* __restrict__ lkeys,
                              unsigned long long* __restrict__ maxdeg) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t d = row_ptr[v + 1] - row_ptr[v];
    key[v] = (lab[v] << 8) | (int32_t)(d < 255 ? d : 255);
    lkeys[v] = ((uint64_t)(uint32_t)lab[v] << 32) | (uint64_t)v;
    atomicMax(maxdeg, (unsigned long long)d);
}

__global__ void k_label_bounds(const uint64_t* __restrict__ lkeys, int64_t n, int64_t L,
                               int64_t* __restrict__ lab_ptr, int32_t* __restrict__ lab_vtx) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    int64_t hi = (p < n) ? (int64_t)(lkeys[p] >> 32) : L;
    int64_t lo = (p == 0) ? -1 : (int64_t)(lkeys[p - 1] >> 32);
    for (int64_t l = lo + 1; l <= hi; l++) lab_ptr[l] = p;
    if (p < n) lab_vtx[p] = (int32_t)(lkeys[p] & 0xFFFFFFFFu);
}

__global__ void k_label_degsum(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ lab, int64_t n,
                               unsigned long long* __restrict__ sum) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) atomicAdd(&sum[lab[v]], (unsigned long long)(row_ptr[v + 1] - row_ptr[v]));
}

// ------------------------------------------------------------ label runs

// kept holds (src << 32 | dst), sorted; rewrite each as (src, label(dst),
// dst) packed into sh_src / sh_lab / 0 bit offsets
__global__ void k_group_keys(uint64_t* __restrict__ kept, int64_t nadj, const int32_t* __restrict__ label,
                             int sh_lab, int sh_src) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nadj) return;
    uint64_t k = kept[i];
    uint64_t src = k >> 32, dst = k & 0xFFFFFFFFull;
    kept[i] = (src << sh_src) | ((uint64_t)(uint32_t)label[dst] << sh_lab) | dst;
}

// back to (src << 32 | dst), now in (src, label, dst) order
__global__ void k_ungroup_keys(uint64_t* __restrict__ kept, int64_t nadj, int sh_src, uint64_t dst_mask) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nadj) return;
    uint64_t k = kept[i];
    kept[i] = ((k >> sh_src) << 32) | (k & dst_mask);
}

// warp per row: number of label runs (write = 0), or the runs themselves
template <bool WRITE>
__global__ void k_row_runs(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ label, int64_t n, int64_t* __restrict__ cnt,
                           const int64_t* __restrict__ run_ptr, int32_t* __restrict__ run_lab,
                           int64_t* __restrict__ run_beg) {
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w; v < n; v += nw) {
        const int64_t a = row_ptr[v], b = row_ptr[v + 1];
        int64_t r = WRITE ? run_ptr[v] : 0;
        int64_t c = 0;
        for (int64_t base = a; base < b; base += 32) {
            int64_t i = base + lane;
            bool head = false;
            int32_t l = 0;
            if (i < b) {
                l = label[col[i]];
                head = (i == a) || label[col[i - 1]] != l;
            }
            uint32_t m = __ballot_sync(0xffffffffu, head);
            if (WRITE && head) {
                int64_t at = r + __popc(m & lanemask_lt());
                run_lab[at] = l;
                run_beg[at] = i;
            }
            r += __popc(m);
            c += __popc(m);
        }
        if (!WRITE && lane == 0) cnt[v] = c;
    }
}

// Adjacency entries per (label of the row's vertex, label of the
// neighbour), M[a * L + b], from the label runs; counted in shared memory
// when the L x L table fits there.
constexpr int kPairSmem = 4096;

__global__ void k_label_pairs(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ run_ptr,
                              const int32_t* __restrict__ run_lab, const int64_t* __restrict__ run_beg,
                              const int32_t* __restrict__ label, int64_t n, int L, unsigned long long* __restrict__ M) {
    extern __shared__ unsigned long long pair_sm[];
    const bool local = L * L <= kPairSmem;
    if (local)
        for (int i = threadIdx.x; i < L * L; i += blockDim.x) pair_sm[i] = 0;
    __syncthreads();
    unsigned long long* dst = local ? pair_sm : M;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = label[v];
        const int64_t r1 = run_ptr[v + 1], end = row_ptr[v + 1];
        for (int64_t r = run_ptr[v]; r < r1; r++) {
            const int64_t len = (r + 1 < r1 ? run_beg[r + 1] : end) - run_beg[r];
            atomicAdd(dst + a * L + run_lab[r], (unsigned long long)len);
        }
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < L * L; i += blockDim.x)
            if (pair_sm[i]) atomicAdd(M + i, pair_sm[i]);
}

int label_pair_counts(fast_graph* g, cudaStream_t s) {
    const int L = g->num_labels;
    if (!g->grouped || L <= 0 || L > kLabelPairMax) return FAST_OK;
    unsigned long long* M = nullptr;
    FAST_TRY(dalloc(&M, (int64_t)L * L, s));
    cudaMemsetAsync(M, 0, (size_t)L * L * sizeof(unsigned long long), s);
    const bool local = L * L <= kPairSmem;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n, 256), (int64_t)num_sms() * 4));
    k_label_pairs<<<blocks, 256, local ? (size_t)L * L * sizeof(unsigned long long) : 0, s>>>(
        g->row_ptr, g->run_ptr, g->run_lab, g->run_beg, g->label, g->n, L, M);
    note_launch();
    std::vector<int64_t> h((size_t)L * L);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), M, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(M, s);
    if (e != cudaSuccess) return cuda_status(e, "label pair counts", __FILE__, __LINE__);
    g->lab_pair_host.swap(h);
    return FAST_OK;
}

int build_label_runs(fast_graph* g, cudaStream_t s) {
    const int64_t n = g->n;
    int64_t* cnt = nullptr;
    FAST_TRY(dalloc(&g->run_ptr, n + 1, s));
    FAST_TRY(dalloc(&cnt, n, s));
    unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n, 8), (int64_t)num_sms() * 32);
    k_row_runs<false><<<blocks, 256, 0, s>>>(g->row_ptr, g->col, g->label, n, cnt, nullptr, nullptr, nullptr);
    note_launch();
    int rc = scan_exclusive<int64_t>(cnt, g->run_ptr, n, g->run_ptr + n, s);
    int64_t R = 0;
    if (rc == FAST_OK) {
        cudaError_t e = cudaMemcpyAsync(&R, g->run_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "label runs", __FILE__, __LINE__);
    }
    dfree(cnt, s);
    if (rc == FAST_OK) rc = dalloc(&g->run_lab, R, s);
    if (rc == FAST_OK) rc = dalloc(&g->run_beg, R, s);
    if (rc == FAST_OK) {
        k_row_runs<true><<<blocks, 256, 0, s>>>(g->row_ptr, g->col, g->label, n, nullptr, g->run_ptr, g->run_lab,
                                                g->run_beg);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "label runs launch");
    }
    if (rc == FAST_OK) g->grouped = true;
    return rc;
}

void graph_release(fast_graph* g, cudaStream_t s) {
    if (!g) return;
    dfree(g->row_ptr, s); dfree(g->col, s); dfree(g->label, s); dfree(g->key, s);
    dfree(g->lab_ptr, s); dfree(g->lab_vtx, s);
    dfree(g->run_ptr, s); dfree(g->run_lab, s); dfree(g->run_beg, s);
    delete g;
}

int load_graph(int64_t n, int64_t m, const int32_t* edges, const int32_t* labels, int flags,
               cudaStream_t s, fast_graph** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_load_graph: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7FFFFFFFll) return set_error(FAST_ERR_INVALID, "fast_load_graph: n=%lld out of range", (long long)n);
    if (m < 0 || 2 * m >= 0xFFFFFFFFll) return set_error(FAST_ERR_INVALID, "fast_load_graph: m=%lld out of range", (long long)m);
    if ((m > 0 && !edges) || !labels) return set_error(FAST_ERR_INVALID, "fast_load_graph: NULL input");
    fast_graph* g = new fast_graph();
    g->n = n;
    int32_t* d_edges = nullptr;
    uint64_t* keys = nullptr;
    uint64_t* kept = nullptr;
    int* flags_d = nullptr;
    uint64_t* lkeys = nullptr;
    unsigned long long* maxdeg_d = nullptr;
    int rc = FAST_OK;
    const bool dev = (flags & FAST_PTR_DEVICE) != 0;
    do {
        rc = dalloc(&g->label, n, s); if (rc) break;
        if (dev) {
            if (cudaMemcpyAsync(g->label, labels, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "label copy"); break; }
        } else {
            if (cudaMemcpyAsync(g->label, labels, n * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "label upload"); break; }
        }
        const int32_t* e_dev = edges;
        if (!dev && m > 0) {
            rc = dalloc(&d_edges, 2 * m, s); if (rc) break;
            if (cudaMemcpyAsync(d_edges, edges, 2 * m * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "edge upload"); break; }
            e_dev = d_edges;
        }
        rc = dalloc(&flags_d, 2, s); if (rc) break;
        cudaMemsetAsync(flags_d, 0, 2 * sizeof(int), s);
        int nb = bits_for(n - 1 > 0 ? n - 1 : 1);
        uint64_t mask = (nb >= 32) ? 0xFFFFFFFFull : ((1ull << nb) - 1);
        uint64_t sent = (mask << 32) | mask;
        rc = dalloc(&keys, 2 * m, s); if (rc) break;
        if (m > 0) { k_edge_keys<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(e_dev, m, n, sent, keys, flags_d); note_launch(); }
        k_check_labels<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(g->label, n, flags_d, flags_d + 1);
        note_launch();
        int hflags[2] = {0, 0};
        if (cudaMemcpyAsync(hflags, flags_d, sizeof(hflags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "loader validation"); break; }
        if (hflags[0] & 1) { rc = set_error(FAST_ERR_INVALID, "fast_load_graph: edge endpoint outside 0..n-1"); break; }
        if (hflags[0] & 2) { rc = set_error(FAST_ERR_INVALID, "fast_load_graph: label outside 0..2^23-1"); break; }
        g->num_labels = hflags[1] + 1;
        int shifts[16];
        int np = digit_shifts(0, nb, shifts, 8);
        np += digit_shifts(32, 32 + nb, shifts + np, 8);
        rc = radix_sort_u64(keys, 2 * m, shifts, np, s); if (rc) break;
        DedupF f{keys, sent};
        int64_t nadj = 0;
        rc = compact_alloc(f, 2 * m, &kept, &nadj, s); if (rc) break;
        g->nadj = nadj;
        dfree(keys, s);
        dfree(d_edges, s);
        // group each row by neighbour label: (src, label, dst) keys, a stable
        // sort on the src and label digits keeps dst ascending within a group
        const int lbits = bits_for(g->num_labels - 1 > 0 ? g->num_labels - 1 : 1);
        const bool group = 2 * nb + lbits <= 64 && nadj > 0;
        if (group) {
            k_group_keys<<<(unsigned)ceil_div(nadj, 256), 256, 0, s>>>(kept, nadj, g->label, nb, nb + lbits);
            note_launch();
            np = digit_shifts(nb, 2 * nb + lbits, shifts, 16);
            rc = radix_sort_u64(kept, nadj, shifts, np, s); if (rc) break;
            k_ungroup_keys<<<(unsigned)ceil_div(nadj, 256), 256, 0, s>>>(kept, nadj, nb + lbits, mask);
            note_launch();
        }
        rc = dalloc(&g->row_ptr, n + 1, s); if (rc) break;
        rc = dalloc(&g->col, nadj, s); if (rc) break;
        k_row_bounds<<<(unsigned)ceil_div(nadj + 1, 256), 256, 0, s>>>(kept, nadj, n, g->row_ptr, g->col);
        note_launch();
        dfree(kept, s);
        if (group) { rc = build_label_runs(g, s); if (rc) break; }
        rc = dalloc(&g->key, n, s); if (rc) break;
        rc = dalloc(&lkeys, n, s); if (rc) break;
        rc = dalloc(&maxdeg_d, 1, s); if (rc) break;
        cudaMemsetAsync(maxdeg_d, 0, sizeof(unsigned long long), s);
        k_vertex_keys<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(g->row_ptr, g->label, n, g->key, lkeys, maxdeg_d);
        note_launch();
        int lb = bits_for(g->num_labels - 1 > 0 ? g->num_labels - 1 : 1);
        np = digit_shifts(32, 32 + lb, shifts, 8);
        rc = radix_sort_u64(lkeys, n, shifts, np, s); if (rc) break;
        rc = dalloc(&g->lab_ptr, g->num_labels + 1, s); if (rc) break;
        rc = dalloc(&g->lab_vtx, n, s); if (rc) break;
        k_label_bounds<<<(unsigned)ceil_div(n + 1, 256), 256, 0, s>>>(lkeys, n, g->num_labels, g->lab_ptr, g->lab_vtx);
        note_launch();
        {
            unsigned long long* ds = nullptr;
            rc = dalloc(&ds, g->num_labels, s); if (rc) break;
            cudaMemsetAsync(ds, 0, g->num_labels * sizeof(unsigned long long), s);
            k_label_degsum<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(g->row_ptr, g->label, n, ds);
            note_launch();
            g->lab_degsum_host.resize(g->num_labels);
            cudaError_t e = cudaMemcpyAsync(g->lab_degsum_host.data(), ds, g->num_labels * sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            dfree(ds, s);
            if (e != cudaSuccess) { rc = cuda_status(e, "label degree sums", __FILE__, __LINE__); break; }
        }
        rc = label_pair_counts(g, s); if (rc) break;
        g->lab_ptr_host.resize(g->num_labels + 1);
        unsigned long long md = 0;
        if (cudaMemcpyAsync(g->lab_ptr_host.data(), g->lab_ptr, (g->num_labels + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&md, maxdeg_d, sizeof(md), cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "label index readback"); break; }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_status(e, "fast_load_graph", __FILE__, __LINE__); break; }
        g->max_degree = (int64_t)md;
    } while (0);
    dfree(d_edges, s); dfree(keys, s); dfree(kept, s); dfree(flags_d, s); dfree(lkeys, s); dfree(maxdeg_d, s);
    if (rc != FAST_OK) {
        graph_release(g, s);
        return rc;
    }
    *out = g;
    return FAST_OK;
}

}  // namespace

extern "C" int fast_load_graph(int64_t n, int64_t m, const int32_t* edges, const int32_t* labels, int flags,
                               void* stream, fast_graph** out) {
    return load_graph(n, m, edges, labels, flags, (cudaStream_t)stream, out);
}

extern "C" int fast_graph_info(const fast_graph* g, int64_t* n, int64_t* nadj, int32_t* num_labels,
                               int64_t* max_degree) {
    if (!g) return set_error(FAST_ERR_INVALID, "fast_graph_info: NULL graph");
    if (n) *n = g->n;
    if (nadj) *nadj = g->nadj;
    if (num_labels) *num_labels = g->num_labels;
    if (max_degree) *max_degree = g->max_degree;
    return FAST_OK;
}

extern "C" int fast_graph_copy_csr(const fast_graph* g, int64_t* row_ptr, int32_t* col, void* stream) {
    if (!g || !row_ptr || (!col && g->nadj)) return set_error(FAST_ERR_INVALID, "fast_graph_copy_csr: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    FAST_CUDA(cudaMemcpyAsync(row_ptr, g->row_ptr, (g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (g->nadj) FAST_CUDA(cudaMemcpyAsync(col, g->col, g->nadj * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    return FAST_OK;
}

extern "C" void fast_free_graph(fast_graph* g) {
    if (!g) return;
    graph_release(g, nullptr);
    cudaStreamSynchronize(nullptr);
    trim_freed_memory();                 // a workload ended: hand its pooled memory back
}
