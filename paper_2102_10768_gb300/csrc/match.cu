// Enumeration over the CST (the semantics of Algorithms 4-8, Sec. V-A).
//
// One warp owns one chunk at a time (a persistent grid pulls chunk indices
// from a global counter) and walks its search space depth first.  Per depth
// the warp scans the candidate list of the parent position's image 32
// entries at a time -- the Generator -- and each lane tests its candidate:
//   EdgeValidator    binary search of the candidate in the CST list of every
//                    earlier non-tree neighbour's image;
//   VisitedValidator the candidate's data vertex against the images of the
//                    earlier positions with the same label (distinct labels
//                    cannot collide);
// a ballot keeps the survivors -- the Synchronizer -- which are buffered in
// shared memory and expanded one by one, or counted (and optionally written
// out) at the last position.  The per-depth scan state lives in registers of
// the lane whose index is the depth (depth <= 31), so no per-depth array is
// indexed dynamically.
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "prims.cuh"

using namespace fast;

namespace {

thread_local double g_last_match_ms = 0.0;

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = false;
    EventPair() {
        ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
};

EventPair& match_events() {
    static thread_local EventPair ev;
    return ev;
}

struct MatchPlan {
    int k;
    int order[kMaxK];                 // position -> query vertex
    int par[kMaxK];                   // position -> parent position
    uint32_t same_lab[kMaxK];         // earlier positions with the same label
    const int32_t* cand[kMaxK];       // by position
    const int64_t* t_off[kMaxK];      // by position (tree edge into it)
    const uint32_t* t_idx[kMaxK];
    int nt_begin[kMaxK + 1];          // non-tree edges into position i
    int nt_from[kMaxNT];              // their earlier endpoint (position)
    const int64_t* n_off[kMaxNT];
    const uint32_t* n_idx[kMaxNT];
};

enum : int { kStatusTimeout = 1, kStatusOverflow = 2 };

struct MatchOut {
    unsigned long long* next_chunk;
    unsigned long long* total;
    unsigned long long* emb_slot;
    int* status;
    uint64_t* chunk_counts;           // nullable
    uint32_t* emb;                    // nullable
    uint64_t emb_cap;
    unsigned long long* stats;        // nullable: [k+1]
    const unsigned long long* deadline;  // device word: %globaltimer limit, 0 = none
};

__global__ void k_set_deadline(unsigned long long* d, unsigned long long budget_ns) {
    *d = budget_ns ? global_timer_ns() + budget_ns : 0ull;
}

__device__ __forceinline__ bool bsearch_u32(const uint32_t* __restrict__ a, int64_t lo, int64_t hi, uint32_t x) {
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo < end && __ldg(a + lo) == x;
}

template <bool STATS, bool EMIT>
__global__ void __launch_bounds__(256) k_match(const MatchPlan P, const Chunk* __restrict__ chunks, int64_t nchunks,
                                               MatchOut O) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t* sbuf = smem + (size_t)warp * (kMaxK * 32 + 2 * kMaxK);   // [depth][32]
    uint32_t* sm = sbuf + kMaxK * 32;                                   // m[position]
    int32_t* sg = (int32_t*)(sm + kMaxK);                               // data vertex per position
    const int k = P.k;
    unsigned long long iter = 0;
    const unsigned long long deadline = *O.deadline;

    for (;;) {
        unsigned long long ci = 0;
        if (lane == 0) {
            ci = (*(volatile int*)O.status & kStatusTimeout) ? (unsigned long long)nchunks : atomicAdd(O.next_chunk, 1ull);
            if (deadline && global_timer_ns() > deadline) { atomicOr(O.status, kStatusTimeout); ci = nchunks; }
        }
        ci = __shfl_sync(0xffffffffu, ci, 0);
        if (ci >= (unsigned long long)nchunks) break;
        const Chunk& ch = chunks[ci];
        const int j = ch.j;
        uint32_t m_reg = lane < j ? ch.prefix[lane] : 0u;      // lane p: candidate index of position p
        int32_t g_reg = -1;                                    // lane p: data vertex of position p
        if (lane < j) g_reg = P.cand[lane][m_reg];
        sm[lane] = m_reg;
        sg[lane] = g_reg;
        __syncwarp();
        unsigned long long bytes = 0;
        // ---- the prefix must itself be a partial embedding (non-tree edges, injectivity)
        bool ok_prefix = true;
        if (lane < j && lane > 0) {
            for (int e = P.nt_begin[lane]; e < P.nt_begin[lane + 1]; e++) {
                uint32_t mf = sm[P.nt_from[e]];
                int64_t lo = P.n_off[e][mf], hi = P.n_off[e][mf + 1];
                if (STATS) bytes += 8 + 4 * (hi - lo);
                if (!bsearch_u32(P.n_idx[e], lo, hi, m_reg)) ok_prefix = false;
            }
            uint32_t sl = P.same_lab[lane];
            while (sl) {
                int p = __ffs(sl) - 1;
                sl &= sl - 1;
                if (sg[p] == g_reg) ok_prefix = false;
            }
        }
        if (STATS) {
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
        }
        unsigned long long count = 0;
        if (__all_sync(0xffffffffu, ok_prefix)) {
            // ---- depth j: the chunk's run of L_j
            int d = j;
            int64_t seg_next = 0, seg_end = 0;     // lane d: scan position in depth d's list
            uint32_t bcnt = 0, bcur = 0;           // lane d: buffered survivors of depth d
            {
                int64_t lo, hi;
                if (j == 0) { lo = ch.a; hi = ch.b; }
                else {
                    uint32_t mp = __shfl_sync(0xffffffffu, m_reg, P.par[j]);
                    int64_t base = P.t_off[j][mp];
                    lo = base + ch.a; hi = base + ch.b;
                }
                if (lane == d) { seg_next = lo; seg_end = hi; }
                if (STATS && lane == 0) {
                    if (j == 0) bytes += 4 * (hi - lo);
                    else {
                        bytes += 8 + 4 * (hi - lo);
                        for (int e = P.nt_begin[j]; e < P.nt_begin[j + 1]; e++) {
                            uint32_t mf = sm[P.nt_from[e]];
                            bytes += 8 + 4 * (P.n_off[e][mf + 1] - P.n_off[e][mf]);
                        }
                    }
                }
            }
            for (;;) {
                if (deadline && ((++iter & 1023) == 0)) {
                    int stop = 0;
                    if (lane == 0) {
                        if (global_timer_ns() > deadline) atomicOr(O.status, kStatusTimeout);
                        stop = *(volatile int*)O.status & kStatusTimeout;
                    }
                    if (__shfl_sync(0xffffffffu, stop, 0)) break;
                }
                uint32_t cur_d = __shfl_sync(0xffffffffu, bcur, d);
                uint32_t cnt_d = __shfl_sync(0xffffffffu, bcnt, d);
                if (cur_d < cnt_d) {
                    // expand the next buffered survivor of depth d
                    uint32_t v = sbuf[d * 32 + cur_d];
                    if (lane == d) { bcur++; m_reg = v; g_reg = P.cand[d][v]; }
                    if (lane == d) { sm[d] = v; sg[d] = g_reg; }
                    d++;
                    uint32_t mp = __shfl_sync(0xffffffffu, m_reg, P.par[d]);
                    int64_t lo = P.t_off[d][mp], hi = P.t_off[d][mp + 1];
                    if (lane == d) { seg_next = lo; seg_end = hi; bcnt = 0; bcur = 0; }
                    __syncwarp();
                    if (STATS && lane == 0) {
                        bytes += 8 + 4 * (hi - lo);
                        for (int e = P.nt_begin[d]; e < P.nt_begin[d + 1]; e++) {
                            uint32_t mf = sm[P.nt_from[e]];
                            bytes += 8 + 4 * (P.n_off[e][mf + 1] - P.n_off[e][mf]);
                        }
                    }
                    continue;
                }
                int64_t sn = __shfl_sync(0xffffffffu, seg_next, d);
                int64_t se = __shfl_sync(0xffffffffu, seg_end, d);
                if (sn < se) {
                    // Generator: next 32 entries of depth d's list
                    int64_t idx = sn + lane;
                    bool ok = idx < se;
                    uint32_t cnd = 0;
                    if (ok) cnd = (d == 0) ? (uint32_t)idx : __ldg(P.t_idx[d] + idx);
                    // EdgeValidator
                    for (int e = P.nt_begin[d]; e < P.nt_begin[d + 1]; e++) {
                        uint32_t mf = __shfl_sync(0xffffffffu, m_reg, P.nt_from[e]);
                        int64_t lo = P.n_off[e][mf], hi = P.n_off[e][mf + 1];
                        if (ok) ok = bsearch_u32(P.n_idx[e], lo, hi, cnd);
                    }
                    // VisitedValidator
                    int32_t gc = -1;
                    uint32_t sl = P.same_lab[d];
                    if (sl || (EMIT && d == k - 1)) {
                        if (ok) gc = __ldg(P.cand[d] + cnd);
                        while (sl) {
                            int p = __ffs(sl) - 1;
                            sl &= sl - 1;
                            int32_t gp = __shfl_sync(0xffffffffu, g_reg, p);
                            if (gp == gc) ok = false;
                        }
                    }
                    // Synchronizer
                    uint32_t mask = __ballot_sync(0xffffffffu, ok);
                    if (lane == d) seg_next = sn + 32;
                    if (STATS && lane == 0) atomicAdd(&O.stats[1 + d], (unsigned long long)__popc(mask));
                    if (d == k - 1) {
                        count += __popc(mask);
                        if (EMIT && mask) {
                            unsigned long long base = 0;
                            if (lane == 0) base = atomicAdd(O.emb_slot, (unsigned long long)__popc(mask));
                            base = __shfl_sync(0xffffffffu, base, 0);
                            unsigned long long slot = base + __popc(mask & lanemask_lt());
                            bool wr = ok && slot < O.emb_cap;
                            for (int p = 0; p < k - 1; p++) {
                                int32_t gp = __shfl_sync(0xffffffffu, g_reg, p);
                                if (wr) O.emb[slot * k + P.order[p]] = (uint32_t)gp;
                            }
                            if (wr) O.emb[slot * k + P.order[k - 1]] = (uint32_t)gc;
                        }
                    } else {
                        if (ok) sbuf[d * 32 + __popc(mask & lanemask_lt())] = cnd;
                        if (lane == d) { bcnt = __popc(mask); bcur = 0; }
                        __syncwarp();
                    }
                    continue;
                }
                // depth d exhausted: backtrack
                if (d == j) break;
                d--;
            }
        }
        if (lane == 0) {
            if (O.chunk_counts) O.chunk_counts[ci] = count;
            if (count) {
                unsigned long long old = atomicAdd(O.total, count);
                if (old + count < old) atomicOr(O.status, kStatusOverflow);
            }
            if (STATS) atomicAdd(&O.stats[0], bytes);
        }
        __syncwarp();
    }
}

MatchPlan make_plan(const fast_cst* c) {
    MatchPlan P;
    memset(&P, 0, sizeof(P));
    int k = c->k;
    P.k = k;
    for (int i = 0; i < k; i++) {
        int u = c->order[i];
        P.order[i] = u;
        P.par[i] = c->parent[u] < 0 ? 0 : c->pos[c->parent[u]];
        P.cand[i] = c->cand[u];
        P.t_off[i] = c->t_off[u];
        P.t_idx[i] = c->t_idx[u];
        P.same_lab[i] = 0;
        for (int p = 0; p < i; p++)
            if (c->qlabel[c->order[p]] == c->qlabel[u]) P.same_lab[i] |= 1u << p;
    }
    int e = 0;
    for (int i = 0; i < k; i++) {
        P.nt_begin[i] = e;
        for (int t = 0; t < c->nnt; t++) {
            if (c->pos[c->nt_to[t]] != i) continue;
            P.nt_from[e] = c->pos[c->nt_from[t]];
            P.n_off[e] = c->n_off[t];
            P.n_idx[e] = c->n_idx[t];
            e++;
        }
    }
    P.nt_begin[k] = e;
    return P;
}

size_t smem_bytes(int warps) { return (size_t)warps * (kMaxK * 32 + 2 * kMaxK) * sizeof(uint32_t); }

int run_match(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg_in, uint64_t kemb, uint32_t* emb_out,
              uint64_t* count_out, uint64_t* written_out, uint64_t* chunk_counts, uint64_t* stats_out,
              cudaStream_t s) {
    if (!c) return set_error(FAST_ERR_INVALID, "fast_match: cst is NULL");
    if (kemb > 0 && !emb_out) return set_error(FAST_ERR_INVALID, "fast_match: k > 0 needs emb_out");
    if (chunks && chunks->c != c) return set_error(FAST_ERR_INVALID, "fast_match: chunks belong to another CST");
    fast_config cfg = cfg_in ? *cfg_in : c->cfg;
    int warps = cfg.warps_per_block > 0 ? cfg.warps_per_block : 8;
    if (warps > 8) warps = 8;
    int bps = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : 4;
    MatchPlan P = make_plan(c);
    Chunk* own = nullptr;
    const Chunk* dchunks = nullptr;
    int64_t nchunks = 0;
    int rc = FAST_OK;
    std::vector<Chunk> roots;
    if (chunks) { dchunks = chunks->d; nchunks = chunks->n; }
    else if (c->ncand[c->root] > 0) {
        // the whole tree: the root's candidates cut into even runs, a few per warp
        uint64_t nr = (uint64_t)c->ncand[c->root];
        uint64_t parts = std::min<uint64_t>(nr, (uint64_t)num_sms() * bps * warps * 4);
        roots.resize(parts);
        for (uint64_t i = 0; i < parts; i++) {
            Chunk& r0 = roots[i];
            memset(&r0, 0, sizeof(r0));
            r0.j = 0; r0.a = (uint32_t)(i * nr / parts); r0.b = (uint32_t)((i + 1) * nr / parts);
        }
        FAST_TRY(dalloc(&own, parts, s));
        cudaError_t e = cudaMemcpyAsync(own, roots.data(), parts * sizeof(Chunk), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { dfree(own, s); return cuda_status(e, "fast_match chunk", __FILE__, __LINE__); }
        dchunks = own; nchunks = (int64_t)parts;
    }
    // counters: [0] next chunk, [1] total, [2] embedding slot, [3] status,
    // [4 .. 4+k] stats, [4+kMaxK+1] deadline
    unsigned long long* ctr = nullptr;
    const int nctr = 4 + kMaxK + 2;
    rc = dalloc(&ctr, nctr, s);
    uint32_t* emb_dev = emb_out;
    uint32_t* staged = nullptr;
    bool timed = false;
    if (rc == FAST_OK && kemb > 0) {
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, emb_out);
        cudaGetLastError();
        bool device_ok = e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        if (!device_ok) {
            rc = dalloc(&staged, kemb * (uint64_t)c->k, s);
            emb_dev = staged;
        }
    }
    if (rc == FAST_OK) {
        cudaMemsetAsync(ctr, 0, nctr * sizeof(unsigned long long), s);
        MatchOut O;
        O.next_chunk = ctr; O.total = ctr + 1; O.emb_slot = ctr + 2; O.status = (int*)(ctr + 3);
        O.chunk_counts = chunk_counts; O.emb = emb_dev; O.emb_cap = kemb;
        O.stats = stats_out ? ctr + 4 : nullptr;
        O.deadline = ctr + 4 + kMaxK + 1;
        unsigned long long budget_ns = cfg.time_budget_s > 0 ? (unsigned long long)(cfg.time_budget_s * 1e9) : 0ull;
        if (budget_ns) { k_set_deadline<<<1, 1, 0, s>>>(ctr + 4 + kMaxK + 1, budget_ns); note_launch(); }
        if (nchunks > 0) {
            int64_t grid = (int64_t)num_sms() * bps;
            grid = std::max<int64_t>(1, std::min<int64_t>(grid, ceil_div(nchunks, warps)));
            size_t sh = smem_bytes(warps);
            EventPair& ev = match_events();
            if (ev.ok) cudaEventRecord(ev.a, s);
            if (stats_out) { k_match<true, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, dchunks, nchunks, O); note_launch(); }
            else if (kemb > 0) { k_match<false, true><<<(unsigned)grid, warps * 32, sh, s>>>(P, dchunks, nchunks, O); note_launch(); }
            else { k_match<false, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, dchunks, nchunks, O); note_launch(); }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_status(e, "matcher launch", __FILE__, __LINE__);
            if (ev.ok) cudaEventRecord(ev.b, s);
            timed = ev.ok;
        }
    }
    unsigned long long h[nctr];
    memset(h, 0, sizeof(h));
    if (rc == FAST_OK) {
        cudaError_t e = cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_match", __FILE__, __LINE__);
        g_last_match_ms = 0.0;
        if (rc == FAST_OK && timed) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, match_events().a, match_events().b) == cudaSuccess) g_last_match_ms = ms;
            else cudaGetLastError();
        }
    }
    if (rc == FAST_OK && staged) {
        uint64_t rows = std::min<uint64_t>(kemb, h[2]);
        cudaError_t e = rows ? cudaMemcpyAsync(emb_out, staged, rows * c->k * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_match embedding readback", __FILE__, __LINE__);
    }
    dfree(ctr, s); dfree(own, s); dfree(staged, s);
    if (rc != FAST_OK) return rc;
    if (count_out) *count_out = h[1];
    if (written_out) *written_out = std::min<uint64_t>(kemb, h[2]);
    if (stats_out) for (int i = 0; i <= c->k; i++) stats_out[i] = h[4 + i];
    int st = (int)h[3];
    if (st & kStatusTimeout) return set_error(FAST_ERR_TIMEOUT, "fast_match: time budget of %.3f s spent", cfg.time_budget_s);
    if (st & kStatusOverflow) return set_error(FAST_ERR_OVERFLOW, "fast_match: count reached 2^64");
    return FAST_OK;
}

}  // namespace

extern "C" int fast_match(const fast_cst* c, const fast_chunks* chunks, uint64_t k, uint32_t* emb_out,
                          uint64_t* count_out, uint64_t* written_out, void* stream) {
    return run_match(c, chunks, nullptr, k, emb_out, count_out, written_out, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int fast_match_ex(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t k,
                             uint32_t* emb_out, uint64_t* count_out, uint64_t* written_out, uint64_t* chunk_counts,
                             void* stream) {
    return run_match(c, chunks, cfg, k, emb_out, count_out, written_out, chunk_counts, nullptr, (cudaStream_t)stream);
}

extern "C" int fast_match_stats(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t* out,
                                void* stream) {
    if (!out) return set_error(FAST_ERR_INVALID, "fast_match_stats: out is NULL");
    uint64_t cnt = 0;
    return run_match(c, chunks, cfg, 0, nullptr, &cnt, nullptr, nullptr, out, (cudaStream_t)stream);
}

extern "C" double fast_last_match_ms(void) { return g_last_match_ms; }
