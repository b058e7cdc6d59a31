// Batched matching: many queries in one matcher launch.
//
// A fast_batch owns fixed device buffers (per-query plans, the concatenated
// chunk list, counters, the ring of donated runs), so that its matcher
// launch can be captured once as a CUDA graph and replayed for every batch.
// A batch run has three phases:
//   1. a pool of host threads, each with its own CUDA stream and scratch
//      pool, builds the CST (Alg. 1) and the partition (Alg. 2) of the
//      queries concurrently -- their device work overlaps and their host
//      round trips hide each other's latency;
//   2. plans and chunks are gathered into the fixed buffers, every chunk
//      tagged with its query;
//   3. the captured graph runs one persistent matcher launch over all
//      chunks of all queries (work stealing across queries), and the
//      per-query counts come back in one copy.
// An autotuner picks, per query-size class, the partition's delta_w and
// max_chunks (how deep the level-synchronous partition goes before the
// depth-first matcher takes over) and, for the launch, warps per CTA and
// CTAs per SM, by timing batch runs on sample queries.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "prims.cuh"

namespace fast {
size_t match_plan_bytes();
int match_plan_fill(const fast_cst* c, void* host_plan);
void match_plan_set_stride(void* host_plans, int nq, int warp_words);
size_t match_counter_words();
size_t match_chunk_bytes();
int match_batched_enqueue(const void* d_plans, int warp_words, const void* d_chunks, const int64_t* d_nchunks,
                          int max_q, unsigned long long* d_qtotal, int* d_qstop, unsigned long long* d_ctr,
                          void* d_dq, uint32_t* d_dq_state, uint64_t dq_cap, uint64_t limit, double budget_s,
                          int warps, int bps, int validators, cudaStream_t s);
int match_smem_optin(size_t bytes);
int match_status_of(const unsigned long long* h_ctr, uint64_t* bytes, uint64_t* floor);
}  // namespace fast

using namespace fast;

namespace {

constexpr int kClasses = 5;                       // |V(q)| <= 4, 8, 16, 24, 32
constexpr uint64_t kBatchQueue = 1 << 16;         // cells of the ring of donated runs
enum { kStatusTimeout = 1, kStatusOverflow = 2, kStatusLimit = 4 };

int size_class(int k) { return k <= 4 ? 0 : k <= 8 ? 1 : k <= 16 ? 2 : k <= 24 ? 3 : 4; }

}  // namespace

struct fast_batch {
    const fast_graph* g = nullptr;
    int device = 0;
    int max_q = 0;
    int nthreads = 8;
    fast_config base;
    fast_config cls[kClasses];
    std::vector<cudaStream_t> ws;
    size_t psize = 0;
    unsigned char* d_plans = nullptr;
    unsigned char* h_plans = nullptr;     // pinned
    int64_t* h_off = nullptr;             // pinned [max_q + 1]
    int64_t* d_off = nullptr;
    int64_t* d_nchunks = nullptr;
    unsigned char* d_chunks = nullptr;
    int64_t chunk_cap = 0;
    unsigned long long* d_ctr = nullptr;
    unsigned long long* d_qtotal = nullptr;
    unsigned long long* h_qtotal = nullptr; // pinned
    unsigned long long* h_ctr = nullptr;    // pinned
    int* d_qstop = nullptr;
    unsigned char* d_dq = nullptr;
    uint32_t* d_dq_state = nullptr;
    // captured matcher launches, by launch shape (a batch's shared-memory
    // stride takes a few values, so each shape is captured once)
    struct Captured {
        int warp_words, warps, bps, val;
        double budget;
        uint64_t limit, cells;
        unsigned char* chunks;
        cudaGraphExec_t exec;
        int kernels;                      // kernels in the graph (launched per replay)
    };
    std::vector<Captured> graphs;
    cudaGraphExec_t exec = nullptr;       // the one chosen for this run
    int g_kernels = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<ScratchPool*> pools;      // per build thread: scratch of its CSTs and partitions
    double last_build_ms = 0.0, last_match_ms = 0.0;
    uint64_t last_bytes = 0, last_floor = 0;
    int64_t last_chunks = 0;
};

namespace {

__global__ void k_tag_chunks(Chunk* chunks, const int64_t* off, int nq) {
    int64_t total = off[nq];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nq;                      // last q with off[q] <= i
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid;
        }
        chunks[i].pad = (chunks[i].pad & 0xFFu) | ((uint32_t)lo << 8);
    }
}

void batch_release(fast_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (auto& c : b->graphs) cudaGraphExecDestroy(c.exec);
    b->graphs.clear();
    cudaStream_t s = nullptr;
    dfree(b->d_plans, s); dfree(b->d_off, s); dfree(b->d_nchunks, s); dfree(b->d_chunks, s);
    dfree(b->d_ctr, s); dfree(b->d_qtotal, s); dfree(b->d_qstop, s); dfree(b->d_dq, s); dfree(b->d_dq_state, s);
    cudaStreamSynchronize(s);
    if (b->h_plans) cudaFreeHost(b->h_plans);
    if (b->h_off) cudaFreeHost(b->h_off);
    if (b->h_qtotal) cudaFreeHost(b->h_qtotal);
    if (b->h_ctr) cudaFreeHost(b->h_ctr);
    for (auto st : b->ws) cudaStreamDestroy(st);
    for (auto p : b->pools) pool_delete(p);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

int batch_create(const fast_graph* g, const fast_config* cfg, int32_t max_q, int32_t nthreads, fast_batch** out) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_batch_create: out is NULL");
    *out = nullptr;
    if (!g || max_q < 1) return set_error(FAST_ERR_INVALID, "fast_batch_create: bad graph or max_queries");
    if (cfg && (cfg->build_rule < 0 || cfg->build_rule > 2))
        return set_error(FAST_ERR_INVALID, "fast_batch_create: build_rule %d (0, 1 or 2)", cfg->build_rule);
    if (cfg && cfg->refine_rule != 0 && (cfg->refine_rule != 2 || cfg->build_rule < 1))
        return set_error(FAST_ERR_INVALID, "fast_batch_create: refine_rule %d needs 2 and build_rule >= 1",
                         cfg->refine_rule);
    fast_batch* b = new fast_batch();
    cudaGetDevice(&b->device);
    b->g = g;
    b->max_q = max_q;
    b->nthreads = nthreads > 0 ? nthreads : 8;
    if (cfg) b->base = *cfg; else fast_config_default(&b->base);
    for (int c = 0; c < kClasses; c++) b->cls[c] = b->base;
    b->psize = match_plan_bytes();
    cudaStream_t s = nullptr;
    int rc = FAST_OK;
    do {
        b->ws.resize(b->nthreads);
        for (auto& st : b->ws)
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "stream create"); break; }
        if (rc) break;
        for (int w = 0; w < b->nthreads; w++) b->pools.push_back(pool_new());
        rc = dalloc(&b->d_plans, (size_t)max_q * b->psize, s); if (rc) break;
        rc = dalloc(&b->d_off, max_q + 1, s); if (rc) break;
        rc = dalloc(&b->d_nchunks, 1, s); if (rc) break;
        rc = dalloc(&b->d_ctr, match_counter_words(), s); if (rc) break;
        rc = dalloc(&b->d_qtotal, max_q, s); if (rc) break;
        rc = dalloc(&b->d_qstop, max_q, s); if (rc) break;
        rc = dalloc(&b->d_dq, kBatchQueue * match_chunk_bytes(), s); if (rc) break;
        rc = dalloc(&b->d_dq_state, kBatchQueue, s); if (rc) break;
        if (cudaMallocHost((void**)&b->h_plans, (size_t)max_q * b->psize) != cudaSuccess ||
            cudaMallocHost((void**)&b->h_off, (size_t)(max_q + 1) * sizeof(int64_t)) != cudaSuccess ||
            cudaMallocHost((void**)&b->h_qtotal, (size_t)max_q * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost((void**)&b->h_ctr, match_counter_words() * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(FAST_ERR_OOM, "fast_batch_create: pinned host allocation failed");
            break;
        }
        if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "event create"); break; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "fast_batch_create"); break; }
    } while (0);
    if (rc) { batch_release(b); return rc; }
    *out = b;
    return FAST_OK;
}

// (Re)capture the matcher launch as a graph when its shape changed.
int batch_graph(fast_batch* b, int warp_words, const fast_config& lc, cudaStream_t s) {
    const uint64_t cells = lc.queue_cells > 0 ? std::min<uint64_t>((uint64_t)lc.queue_cells, kBatchQueue) : kBatchQueue;
    int warps = lc.warps_per_block > 0 ? std::min(lc.warps_per_block, 8) : 8;
    const int nval = lc.matcher_rule == 1 && warps >= 2 ? (lc.validators > 0 ? std::min(lc.validators, warps - 1) : warps / 2) : 0;
    const int bps = lc.blocks_per_sm > 0 ? lc.blocks_per_sm : 4;
    for (auto& c : b->graphs)
        if (c.warp_words == warp_words && c.warps == warps && c.bps == bps && c.val == nval && c.budget == lc.time_budget_s &&
            c.limit == lc.limit && c.cells == cells && c.chunks == b->d_chunks) {
            b->exec = c.exec;
            b->g_kernels = c.kernels;
            return FAST_OK;
        }
    // a new shape; graphs over an older chunk array can never run again
    for (size_t i = 0; i < b->graphs.size();) {
        if (b->graphs[i].chunks != b->d_chunks) {
            cudaGraphExecDestroy(b->graphs[i].exec);
            b->graphs.erase(b->graphs.begin() + i);
        } else {
            i++;
        }
    }
    if (b->graphs.size() >= 8) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
    }
    FAST_TRY(match_smem_optin((size_t)warps * warp_words * sizeof(uint32_t)));
    cudaStream_t cap;
    FAST_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = FAST_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = cuda_status(e, "begin capture", __FILE__, __LINE__);
    if (rc == FAST_OK) {
        int rc2 = match_batched_enqueue(b->d_plans, warp_words, b->d_chunks, b->d_nchunks, b->max_q, b->d_qtotal,
                                        b->d_qstop, b->d_ctr, b->d_dq, b->d_dq_state, cells, lc.limit,
                                        lc.time_budget_s, warps, bps, nval, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (rc2 != FAST_OK) rc = rc2;
        else if (e != cudaSuccess) rc = cuda_status(e, "end capture", __FILE__, __LINE__);
    }
    if (rc == FAST_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) rc = cuda_status(e, "graph instantiate", __FILE__, __LINE__);
    }
    // the enqueue counted each kernel it recorded (one kernel node each);
    // they run, and are counted, at each replay instead
    int recorded = 0;
    if (rc == FAST_OK) {
        size_t nodes = 0;
        std::vector<cudaGraphNode_t> nv;
        if (cudaGraphGetNodes(graph, nullptr, &nodes) == cudaSuccess) {
            nv.resize(nodes);
            if (nodes && cudaGraphGetNodes(graph, nv.data(), &nodes) != cudaSuccess) nv.clear();
        }
        for (auto nd : nv) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) recorded++;
        }
        cudaGetLastError();
    }
    note_launch(-recorded);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    (void)s;
    if (rc == FAST_OK) {
        b->graphs.push_back({warp_words, warps, bps, nval, lc.time_budget_s, lc.limit, cells, b->d_chunks, exec, recorded});
        b->exec = exec;
        b->g_kernels = recorded;
    } else if (exec) {
        cudaGraphExecDestroy(exec);
    }
    return rc;
}

int batch_run(fast_batch* b, int32_t nq, const fast_query_desc* qs, uint64_t* counts, int32_t* status, cudaStream_t s) {
    if (!b) return set_error(FAST_ERR_INVALID, "fast_batch_run: batch is NULL");
    if (nq < 0 || nq > b->max_q) return set_error(FAST_ERR_INVALID, "fast_batch_run: %d queries (capacity %d)", nq, b->max_q);
    if (nq > 0 && (!qs || !counts || !status)) return set_error(FAST_ERR_INVALID, "fast_batch_run: NULL array");
    std::vector<fast_cst*> csts(nq, nullptr);
    std::vector<fast_chunks*> chs(nq, nullptr);
    std::vector<int32_t> st(nq, FAST_OK);
    auto t0 = std::chrono::steady_clock::now();
    // ---- 1. CSTs and partitions, concurrently (build_rule 1: the CSTs of
    //         all queries together first, then the partitions; 2: the
    //         partitions together too)
    const bool together = b->base.build_rule >= 1;
    const bool parts_together = b->base.build_rule == 2;
    if (together && nq > 0) {
        std::vector<const fast_config*> cf(nq);
        for (int i = 0; i < nq; i++) cf[i] = &b->cls[size_class(qs[i].n)];
        int rc = FAST_OK;
        {
            PoolScope scratch(b->ws[0], b->pools[0]);
            rc = build_cst_batch(b->g, nq, qs, cf.data(), b->ws[0], csts.data(), st.data());
        }
        if (rc == FAST_OK && cudaStreamSynchronize(b->ws[0]) != cudaSuccess)
            rc = set_error(FAST_ERR_CUDA, "fast_batch_run: batched CST build");
        if (rc != FAST_OK) {
            for (int i = 0; i < nq; i++) cst_release_nosync(csts[i]);
            return rc;
        }
    }
    if (parts_together && nq > 0) {
        std::vector<const fast_cst*> cc(nq);
        std::vector<const fast_config*> cf(nq);
        std::vector<int32_t> pst(nq, FAST_OK);
        for (int i = 0; i < nq; i++) {
            cc[i] = st[i] == FAST_OK ? csts[i] : nullptr;
            cf[i] = &b->cls[size_class(qs[i].n)];
        }
        int rc = FAST_OK;
        {
            PoolScope scratch(b->ws[0], b->pools[0]);
            rc = partition_batch(cc.data(), nq, cf.data(), b->ws[0], chs.data(), pst.data());
        }
        if (rc == FAST_OK && cudaStreamSynchronize(b->ws[0]) != cudaSuccess)
            rc = set_error(FAST_ERR_CUDA, "fast_batch_run: batched partition");
        if (rc != FAST_OK) {
            for (int i = 0; i < nq; i++) cst_release_nosync(csts[i]);
            return rc;
        }
    } else {
        std::atomic<int> next{0};
        int T = std::min<int>(b->nthreads, std::max(nq, 1));
        std::vector<std::thread> pool;
        for (int w = 0; w < T; w++) {
            pool.emplace_back([&, w]() {
                cudaSetDevice(b->device);
                PoolScope scratch(b->ws[w], b->pools[w]);
                for (;;) {
                    int i = next.fetch_add(1);
                    if (i >= nq) break;
                    const fast_config& cc = b->cls[size_class(qs[i].n)];
                    int rc = together ? st[i] : fast_build_cst(b->g, &qs[i], &cc, b->ws[w], &csts[i]);
                    if (rc == FAST_OK) rc = fast_partition(csts[i], &cc, b->ws[w], &chs[i]);
                    st[i] = rc;
                }
            });
        }
        for (auto& th : pool) th.join();
    }
    auto t1 = std::chrono::steady_clock::now();
    b->last_build_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    int rc = FAST_OK;
    // ---- 2. gather
    int64_t total = 0;
    int warp_words = 0;
    b->h_off[0] = 0;
    for (int i = 0; i < nq; i++) {
        int64_t n = (st[i] == FAST_OK && chs[i]) ? chs[i]->n : 0;
        b->h_off[i + 1] = b->h_off[i] + n;
        if (st[i] == FAST_OK) warp_words = std::max(warp_words, match_plan_fill(csts[i], b->h_plans + (size_t)i * b->psize));
        else memset(b->h_plans + (size_t)i * b->psize, 0, b->psize);
    }
    total = b->h_off[nq];
    b->last_chunks = total;
    if (warp_words == 0) warp_words = 32 * 32 + 64;
    // one stride for every query of the launch, rounded up to 256 words so
    // that batches of other mixes reuse a captured launch
    warp_words = (warp_words + 255) / 256 * 256;
    match_plan_set_stride(b->h_plans, nq, warp_words);
    do {
        if (total > b->chunk_cap) {
            int64_t cap = std::max<int64_t>(total, 2 * b->chunk_cap);
            dfree(b->d_chunks, s);
            b->chunk_cap = 0;                     // stays 0 if the allocation below fails
            rc = dalloc(&b->d_chunks, (size_t)cap * match_chunk_bytes(), s); if (rc) break;
            b->chunk_cap = cap;
        }
        for (int i = 0; i < nq; i++) {
            int64_t n = b->h_off[i + 1] - b->h_off[i];
            if (n) {
                cudaError_t e = cudaMemcpyAsync(b->d_chunks + b->h_off[i] * match_chunk_bytes(), chs[i]->d,
                                                n * match_chunk_bytes(), cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) { rc = cuda_status(e, "chunk gather", __FILE__, __LINE__); break; }
            }
        }
        if (rc) break;
        if (nq > 0) FAST_CUDA_BREAK(rc, cudaMemcpyAsync(b->d_plans, b->h_plans, (size_t)nq * b->psize, cudaMemcpyHostToDevice, s));
        if (nq > 0) FAST_CUDA_BREAK(rc, cudaMemcpyAsync(b->d_off, b->h_off, (size_t)(nq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        FAST_CUDA_BREAK(rc, cudaMemcpyAsync(b->d_nchunks, &b->h_off[nq], sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (total > 0) {
            k_tag_chunks<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, s>>>((Chunk*)b->d_chunks, b->d_off, nq);
            note_launch();
        }
        // ---- 3. one matcher launch for all queries (captured graph)
        fast_config lc = b->base;
        lc.warps_per_block = b->cls[0].warps_per_block;
        lc.blocks_per_sm = b->cls[0].blocks_per_sm;
        lc.matcher_rule = b->cls[0].matcher_rule;
        lc.validators = b->cls[0].validators;
        rc = batch_graph(b, warp_words, lc, s); if (rc) break;
        FAST_CUDA_BREAK(rc, cudaEventRecord(b->ev0, s));
        FAST_CUDA_BREAK(rc, cudaGraphLaunch(b->exec, s));
        note_launch(b->g_kernels);            // the kernels the graph holds, matcher included
        FAST_CUDA_BREAK(rc, cudaEventRecord(b->ev1, s));
        if (nq > 0) FAST_CUDA_BREAK(rc, cudaMemcpyAsync(b->h_qtotal, b->d_qtotal, (size_t)nq * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        FAST_CUDA_BREAK(rc, cudaMemcpyAsync(b->h_ctr, b->d_ctr, match_counter_words() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_status(e, "fast_batch_run", __FILE__, __LINE__); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        b->last_match_ms = ms;
    } while (0);
    int gst = match_status_of(b->h_ctr, &b->last_bytes, &b->last_floor);
    cudaStreamSynchronize(s);               // no gather copy may still read a chunk list
    for (int i = 0; i < nq; i++) {
        // the matcher is done (or never ran); the builders' streams stay ordered
        chunks_release_nosync(chs[i]);
        cst_release_nosync(csts[i]);
    }
    if (rc != FAST_OK) return rc;
    uint64_t limit = b->base.limit;
    for (int i = 0; i < nq; i++) {
        if (st[i] != FAST_OK) { counts[i] = 0; status[i] = st[i]; continue; }
        uint64_t c = b->h_qtotal[i];
        bool reached = limit && c >= limit;
        counts[i] = reached ? limit : c;
        status[i] = (!reached && (gst & kStatusTimeout)) ? FAST_ERR_TIMEOUT : ((gst & kStatusOverflow) ? FAST_ERR_OVERFLOW : FAST_OK);
    }
    return FAST_OK;
}

}  // namespace

extern "C" int fast_batch_create(const fast_graph* g, const fast_config* cfg, int32_t max_queries, int32_t threads,
                                 fast_batch** out) {
    return batch_create(g, cfg, max_queries, threads, out);
}

extern "C" int fast_batch_run(fast_batch* b, int32_t nq, const fast_query_desc* qs, uint64_t* counts_out,
                              int32_t* status_out, void* stream) {
    return batch_run(b, nq, qs, counts_out, status_out, (cudaStream_t)stream);
}

extern "C" int fast_batch_timing(const fast_batch* b, double* build_ms, double* match_ms, uint64_t* match_bytes,
                                 int64_t* chunks) {
    if (!b) return set_error(FAST_ERR_INVALID, "fast_batch_timing: NULL batch");
    if (build_ms) *build_ms = b->last_build_ms;
    if (match_ms) *match_ms = b->last_match_ms;
    if (match_bytes) *match_bytes = b->last_bytes;
    if (chunks) *chunks = b->last_chunks;
    return FAST_OK;
}

extern "C" int fast_batch_bytes(const fast_batch* b, uint64_t* requested, uint64_t* floor) {
    if (!b) return set_error(FAST_ERR_INVALID, "fast_batch_bytes: NULL batch");
    if (requested) *requested = b->last_bytes;
    if (floor) *floor = b->last_floor;
    return FAST_OK;
}

extern "C" int fast_batch_config(fast_batch* b, int32_t size_class_k, fast_config* get, const fast_config* set) {
    if (!b) return set_error(FAST_ERR_INVALID, "fast_batch_config: NULL batch");
    int c = size_class(size_class_k);
    if (set) b->cls[c] = *set;
    if (get) *get = b->cls[c];
    return FAST_OK;
}

extern "C" int fast_batch_autotune(fast_batch* b, int32_t nq, const fast_query_desc* sample, double* best_ms,
                                   void* stream) {
    if (!b || nq < 1 || !sample) return set_error(FAST_ERR_INVALID, "fast_batch_autotune: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint64_t> cnt(nq);
    std::vector<int32_t> stv(nq);
    // a choice's time: the better of two runs (the first may capture a launch)
    auto timed = [&](int m, const fast_query_desc* q, double* ms) -> int {
        *ms = 1e300;
        for (int rep = 0; rep < 2; rep++) {
            auto t0 = std::chrono::steady_clock::now();
            int rc = batch_run(b, m, q, cnt.data(), stv.data(), s);
            if (rc != FAST_OK) return rc;
            *ms = std::min(*ms, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
        }
        return FAST_OK;
    };
    // per size class: delta_w and max_chunks (chunk size / depth of the BFS phase)
    const uint64_t dws[] = {1ull << 14, 1ull << 17, 1ull << 20, 1ull << 23};
    const int64_t mcs[] = {1024, 4096, 16384};
    double total_best = 0.0;
    for (int c = 0; c < kClasses; c++) {
        std::vector<fast_query_desc> qc;
        for (int i = 0; i < nq; i++) if (size_class(sample[i].n) == c) qc.push_back(sample[i]);
        if (qc.empty()) continue;
        fast_config best = b->cls[c];
        double best_t = 1e300;
        for (uint64_t dw : dws)
            for (int64_t mc : mcs) {
                fast_config trial = b->cls[c];
                trial.delta_w = dw;
                trial.max_chunks = mc;
                b->cls[c] = trial;
                double ms = 0.0;
                FAST_TRY(timed((int)qc.size(), qc.data(), &ms));
                if (ms < best_t) { best_t = ms; best = trial; }
            }
        b->cls[c] = best;
        total_best += best_t;
    }
    // launch shape for the shared matcher launch: warps per CTA, CTAs per SM
    const int shapes[][2] = {{8, 4}, {8, 3}, {8, 2}, {4, 6}};
    double best_t = 1e300;
    int bw = b->cls[0].warps_per_block, bb = b->cls[0].blocks_per_sm;
    for (auto& sh : shapes) {
        for (int c = 0; c < kClasses; c++) { b->cls[c].warps_per_block = sh[0]; b->cls[c].blocks_per_sm = sh[1]; }
        double ms = 0.0;
        FAST_TRY(timed(nq, sample, &ms));
        if (ms < best_t) { best_t = ms; bw = sh[0]; bb = sh[1]; }
    }
    for (int c = 0; c < kClasses; c++) { b->cls[c].warps_per_block = bw; b->cls[c].blocks_per_sm = bb; }
    if (best_ms) *best_ms = best_t;
    (void)total_best;
    return FAST_OK;
}

extern "C" void fast_free_batch(fast_batch* b) { batch_release(b); }

extern "C" int fast_match_batch(const fast_graph* g, int32_t nq, const fast_query_desc* qs, const fast_config* cfg,
                                uint64_t* counts_out, int32_t* status_out, void* stream) {
    fast_batch* b = nullptr;
    FAST_TRY(batch_create(g, cfg, std::max(nq, 1), 0, &b));
    int rc = batch_run(b, nq, qs, counts_out, status_out, (cudaStream_t)stream);
    batch_release(b);
    return rc;
}
