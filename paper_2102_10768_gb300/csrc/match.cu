// Enumeration over the CST (the semantics of Algorithms 4-8, Sec. V-A).
//
// One warp owns one work item at a time -- a chunk of the partition, or a
// run another warp gave away -- and walks its search space depth first.  Per
// depth the warp scans a candidate list 32 entries at a time (the
// Generator) and each lane tests its candidate:
//   Generator        the candidates of depth d are the intersection of the
//                    tree list from the parent's image and the CST list from
//                    every earlier non-tree neighbour's image, all sorted
//                    over C(u_d); the warp scans the shortest of them;
//   EdgeValidator    membership in each other list by a warp-cooperative
//                    merge (a cursor per list, coalesced 32-entry tiles, a
//                    shuffle search, galloping), shortest lists first,
//                    stopping once no candidate is left;
//   VisitedValidator the candidate's data vertex against the images of the
//                    earlier positions with the same label (distinct labels
//                    cannot collide);
// a ballot keeps the survivors (the Synchronizer), which are buffered in
// shared memory and expanded one by one, or counted -- and optionally written
// out -- at the last position.  The per-depth scan state lives in registers
// of the lane whose index is the depth (depth <= 31), so no per-depth array
// is indexed dynamically.
//
// Load balance: a persistent grid first drains the static chunk list, then a
// global ring of donated runs.  A warp that finds both empty counts itself
// idle; a busy warp that sees idle warps gives away the second half of the
// unscanned list at its shallowest depth with at least two entries left --
// a run of a list with a fixed prefix, i.e. again a chunk.  An outstanding-
// work counter ends the launch.  No warp waits on another: the only wait, an
// idle warp looking for work, is bounded by %globaltimer.
//
// Warp-specialised variant (the GPU form of the task-generator separation
// of Sec. V-D): a CTA's warps split into expanders and validators.  The
// expanders run the search above, but a partial result that reaches the
// last position is not scanned there: its extension (the offsets of every
// list into that position, the chosen generator list and the images so
// far) goes into a ring in shared memory as a task, and the expander goes
// on with the next partial result.  Validator warps take tasks and run the
// last position's Generator, EdgeValidator, VisitedValidator and count.
// The last position holds most of the work (hundreds of embeddings per
// partial result on the workloads here), so the expanders' branchy,
// latency-bound descent and the validators' streaming list scans overlap.
// A full ring never blocks an expander: it scans that extension itself.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "prims.cuh"

using namespace fast;

namespace {

thread_local double g_last_match_ms = 0.0;
thread_local uint64_t g_last_match_bytes = 0;
thread_local uint64_t g_last_match_floor = 0;

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
    int warp_words;                   // shared words per warp (survivors, m, data ids, cursors)
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

enum : int { kStatusTimeout = 1, kStatusOverflow = 2, kStatusLimit = 4 };
// shared words per warp: survivors [32 depths][32], m and data vertex per
// position, the generator list of each depth, an 8-byte tree-list cursor per
// depth, then one 8-byte cursor per non-tree edge of the query
constexpr int kWarpBaseWords = kMaxK * 32 + 3 * kMaxK + 2 * kMaxK;
// Chunk.pad: bit 0 = a donated run; bits 1-6 = the list the run belongs to
// (0: the tree list of position j; s: the s-th non-tree edge into j); the
// query of a batch from bit 8 up.
constexpr uint32_t kDonated = 1;
__device__ __forceinline__ int run_source(uint32_t pad) { return (int)((pad >> 1) & 63u); }
constexpr unsigned long long kIdleNs = 5ull * 1000 * 1000 * 1000;     // an idle warp gives up waiting

struct MatchOut {
    unsigned long long* next_chunk;
    unsigned long long* total;        // per query (one entry unless batched)
    int* qstop;                       // per query: limit reached
    int nq;
    unsigned long long* emb_slot;
    int* status;
    uint64_t* chunk_counts;           // nullable (static chunks; no donation then)
    uint32_t* emb;                    // nullable
    uint64_t emb_cap;                 // rows that may be written
    unsigned long long* stats;        // nullable: [k] partial results per depth
    unsigned long long* bytes;        // bytes the search requested
    unsigned long long* floor;        // the floor of those bytes (see k_match)
    const unsigned long long* deadline;  // device word: %globaltimer limit, 0 = none
    uint64_t limit;                   // 0 = enumerate everything
    // Donated runs: a bounded ring of dq_cap cells.  Ticket t (a count of
    // claims, dq_tail for donors and dq_head for takers) uses cell t % dq_cap
    // in generation g = t / dq_cap; the cell's state is 2g while it is free
    // for that ticket and 2g+1 once the run is published; the taker sets
    // 2g+2 after reading it.  States start at 0.  Nobody waits on a cell: a
    // donor that finds its cell still occupied keeps its work, and a taker
    // that finds no published cell looks again later.
    Chunk* dq;
    uint32_t* dq_state;
    uint64_t dq_cap;                  // 0 = no donation
    unsigned long long* dq_head;
    unsigned long long* dq_tail;
    unsigned long long* outstanding;  // work items not yet finished
    unsigned int* idle;               // warps waiting for work
    int validators;                   // warp-specialised variant: validator warps per CTA
};

// One last-position extension handed from an expander to a validator warp
// (the warp-specialised variant): the lists into position k-1 -- index 0
// the tree list, 1 + e the e-th non-tree edge into it -- as index ranges of
// their arrays, which of them generates, and the images of positions
// 0..k-2.
struct VTask {
    uint32_t q;                       // query (batched launches)
    int32_t src;                      // the generator: 0 the tree list, s > 0 non-tree edge s-1
    int64_t lo[kMaxK];
    int64_t hi[kMaxK];
    int32_t g[kMaxK];
};
constexpr int kRing = 8;                          // tasks per CTA
constexpr unsigned long long kValidatorWaitNs = 30ull * 1000 * 1000 * 1000;   // never expected: error after
// the ring's shared words: tickets of producers (tail) and consumers (head),
// per cell a state (2g free for generation g, 2g+1 published), and the
// expanders still running
struct VRing {
    unsigned long long head, tail;
    uint32_t state[kRing];
    int active;
    int pad;
    VTask task[kRing];
};
enum : int { kStatusValidator = 8 };

__global__ void k_set_deadline(unsigned long long* d, unsigned long long budget_ns) {
    *d = budget_ns ? global_timer_ns() + budget_ns : 0ull;
}

__global__ void k_copy_word(unsigned long long* dst, const int64_t* src) { *dst = (unsigned long long)*src; }

// membership of x in the sorted a[lo, hi); *probes counts the entries read
__device__ __forceinline__ bool bsearch_u32(const uint32_t* __restrict__ a, int64_t lo, int64_t hi, uint32_t x,
                                            unsigned long long* probes) {
    int64_t end = hi;
    unsigned long long p = 0;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        p++;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    bool hit = false;
    if (lo < end) { p++; hit = __ldg(a + lo) == x; }
    *probes += p;
    return hit;
}

// Warp-cooperative membership test.  Each lane with `act` holds a candidate
// c; over those lanes the candidates ascend with the lane index (they come
// from the generator list, sorted).  L[0, n) is another sorted list over the
// same candidate set (one CST list: n < 2^31) and *pos a cursor into it that
// never passes the lower bound of any candidate still to come, so successive
// 32-entry segments of the generator walk L once, merge-style:
//   - load the tile L[pos, pos+32) with one coalesced read;
//   - every pending lane whose candidate is <= the tile's last entry finds
//     its lower bound inside the tile by a 5-step shuffle search;
//   - if the smallest pending candidate lies beyond the tile, gallop: lanes
//     probe pos + 32*2^i in one round, then 33-way refinement rounds, each a
//     single parallel read, until a 32-entry window holds its lower bound.
// Returns whether this lane's candidate is in the list; *lb counts the
// entries this lane read (4 B each).
__device__ __forceinline__ bool warp_member(const uint32_t* __restrict__ L, uint32_t n, uint32_t* pos,
                                            uint32_t c, bool act, unsigned long long* lb) {
    const int lane = threadIdx.x & 31;
    bool found = false;
    uint32_t pend = __ballot_sync(0xffffffffu, act);
    uint32_t p0 = *pos;
    uint32_t last = p0;
    while (pend) {
        if (p0 >= n) break;                                // list exhausted: the rest are absent
        int tl = __ffs(pend) - 1;
        uint32_t ct = __shfl_sync(0xffffffffu, c, tl);     // smallest pending candidate
        uint32_t v = 0xFFFFFFFFu;
        if (p0 + lane < n) { v = __ldg(L + p0 + lane); *lb += 4; }
        uint32_t tmax = __shfl_sync(0xffffffffu, v, 31);
        if (tmax < ct) {
            // gallop: the lower bound of ct lies past this (full) tile
            uint32_t a = p0 + 32;                           // first index that may hold it
            uint32_t probe = p0 + 31 + (32u << (lane < 25 ? lane : 25));   // below 2^32: p0 < 2^31
            if (probe > n - 1) probe = n - 1;
            uint32_t pv = __ldg(L + probe);
            *lb += 4;
            uint32_t ge = __ballot_sync(0xffffffffu, pv >= ct);
            if (!ge) { p0 = n; break; }                     // everything left is smaller: all absent
            int f = __ffs(ge) - 1;
            uint32_t b = __shfl_sync(0xffffffffu, probe, f);            // L[b] >= ct
            if (f > 0) a = __shfl_sync(0xffffffffu, probe, f - 1) + 1; // L[a-1] < ct
            while (b - a > 31) {                            // 33-way refinement of [a, b]
                const uint64_t span = b - a + 1;
                uint32_t q = a + (uint32_t)(((uint64_t)(lane + 1) * span) / 33);
                uint32_t qv = __ldg(L + q);
                *lb += 4;
                uint32_t g2 = __ballot_sync(0xffffffffu, qv >= ct);
                int f2 = g2 ? __ffs(g2) - 1 : 32;
                uint32_t nb = f2 < 32 ? __shfl_sync(0xffffffffu, q, f2 < 32 ? f2 : 0) : b;
                uint32_t na = f2 > 0 ? __shfl_sync(0xffffffffu, q, f2 > 0 ? f2 - 1 : 0) + 1 : a;
                a = na;
                b = nb;
            }
            p0 = a;
            continue;
        }
        // resolve every pending lane whose candidate is within this tile
        bool mine = ((pend >> lane) & 1u) && c <= tmax;
        int q = 0;
#pragma unroll
        for (int st = 16; st; st >>= 1) {
            uint32_t w = __shfl_sync(0xffffffffu, v, q + st - 1);
            if (w < c) q += st;
        }
        uint32_t w = __shfl_sync(0xffffffffu, v, q);
        if (mine) found = (w == c);
        pend &= ~__ballot_sync(0xffffffffu, mine);
        last = p0;
        p0 += 32;
    }
    *pos = last;
    return found;
}

__device__ __forceinline__ int vload(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

// lane 0: add a local count to query q's total; flag the limit once reached
__device__ __forceinline__ void flush_count(const MatchOut& O, uint32_t q, unsigned long long& local) {
    if (!local) return;
    unsigned long long old = atomicAdd(&O.total[q], local);
    if (old + local < old) atomicOr(O.status, kStatusOverflow);
    if (O.limit && old + local >= O.limit) {
        O.qstop[q] = 1;
        if (O.nq == 1) atomicOr(O.status, kStatusLimit);
    }
    local = 0;
}

// lane 0: obtain the next work item.  kind 1 = static chunk, 2 = donated run,
// 0 = nothing left (or stop requested).
__device__ int acquire(const MatchOut& O, int64_t nchunks, unsigned long long deadline, unsigned long long* idx) {
    bool was_idle = false;
    int kind = 0;
    unsigned long long t_idle = 0;
    for (;;) {
        if (vload(O.status) & (kStatusTimeout | kStatusLimit)) break;
        unsigned long long now = global_timer_ns();
        if (deadline && now > deadline) { atomicOr(O.status, kStatusTimeout); break; }
        if (vload(O.next_chunk) < (unsigned long long)nchunks) {
            unsigned long long i = atomicAdd(O.next_chunk, 1ull);
            if (i < (unsigned long long)nchunks) { *idx = i; kind = 1; break; }
        }
        if (O.dq_cap) {
            unsigned long long h = vload(O.dq_head);
            uint32_t want = (uint32_t)(2 * (h / O.dq_cap) + 1);          // published, ticket h
            if (*(volatile uint32_t*)&O.dq_state[h % O.dq_cap] == want) {
                if (atomicCAS(O.dq_head, h, h + 1) == h) {
                    __threadfence();
                    *idx = h;
                    kind = 2;
                    break;
                }
                continue;                                                 // taken by another warp
            }
        }
        if (vload(O.outstanding) == 0) break;
        if (!was_idle) { atomicAdd(O.idle, 1u); was_idle = true; t_idle = now; }
        else if (now - t_idle > kIdleNs) break;   // the warps still busy finish (and drain) the rest
        __nanosleep(200);
    }
    if (was_idle) atomicSub(O.idle, 1u);
    return kind;
}

// lane 0: claim the ring's next cell for a producer, if it is free (a cell
// still holding an older task means the ring is full).  Returns the ticket,
// or ~0 when full.
__device__ __forceinline__ unsigned long long ring_claim(VRing* ring) {
    unsigned long long t = *(volatile unsigned long long*)&ring->tail;
    for (int tries = 0; tries < 8; tries++) {
        const uint32_t st = *(volatile uint32_t*)&ring->state[t % kRing];
        if (st == (uint32_t)(2 * (t / kRing))) {
            const unsigned long long prev = atomicCAS(&ring->tail, t, t + 1);
            if (prev == t) return t;
            t = prev;
            continue;
        }
        const unsigned long long now = *(volatile unsigned long long*)&ring->tail;
        if (now == t) break;                                   // full
        t = now;
    }
    return ~0ull;
}

// A validator warp of the warp-specialised matcher: take published tasks
// from the CTA's ring and count the embeddings of their last position --
// the Generator over the chosen list, the EdgeValidator's merges against
// the other lists (cursors in `cur`, one per list), the VisitedValidator
// against the task's images.  Returns once every expander of the CTA has
// left and the ring is empty.  Its bytes go to lb (each lane) and fb (lane
// 0) as the fused search counts them.
template <bool BATCH>
__device__ void validate_tasks(const MatchPlan& P0, const MatchPlan* __restrict__ plans, VRing* ring, int64_t* cur,
                               const MatchOut& O, unsigned long long deadline, unsigned long long& lb,
                               unsigned long long& fb) {
    const int lane = threadIdx.x & 31;
    unsigned long long waited_since = 0;
    for (;;) {
        long long got = -1;
        if (lane == 0) {
            for (;;) {
                unsigned long long h = *(volatile unsigned long long*)&ring->head;
                if (*(volatile uint32_t*)&ring->state[h % kRing] == (uint32_t)(2 * (h / kRing) + 1)) {
                    if (atomicCAS(&ring->head, h, h + 1) == h) { got = (long long)h; break; }
                    continue;
                }
                if (*(volatile int*)&ring->active == 0) {
                    // every expander published its last task before it left: look once more
                    h = *(volatile unsigned long long*)&ring->head;
                    if (*(volatile uint32_t*)&ring->state[h % kRing] == (uint32_t)(2 * (h / kRing) + 1)) continue;
                    got = -2;
                    break;
                }
                const unsigned long long now = global_timer_ns();
                if (!waited_since) waited_since = now;
                else if (now - waited_since > kValidatorWaitNs) { atomicOr(O.status, kStatusValidator); got = -2; break; }
                __nanosleep(2000);
            }
            __threadfence_block();
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got < 0) return;
        waited_since = 0;
        __syncwarp();
        const VTask& T = ring->task[got % kRing];
        const uint32_t q = T.q;
        const MatchPlan& P = BATCH ? plans[q] : P0;
        const int d = P.k - 1;
        const int e0 = P.nt_begin[d], ne = P.nt_begin[d + 1] - e0;
        const int src = T.src;
        const int64_t glo = T.lo[src], ghi = T.hi[src];
        const uint32_t* gen = src == 0 ? P.t_idx[d] : P.n_idx[e0 + src - 1];
        if (lane <= ne) cur[lane] = 0;
        __syncwarp();
        unsigned long long local = 0;
        int it = 0;
        bool stop = false;
        for (int64_t sn = glo; sn < ghi && !stop; sn += 32) {
            if ((++it & 255) == 0) {
                int st = 0;
                if (lane == 0) {
                    flush_count(O, q, local);
                    if (deadline && global_timer_ns() > deadline) atomicOr(O.status, kStatusTimeout);
                    st = vload(O.status) & (kStatusTimeout | kStatusLimit);
                    if (BATCH && *(volatile int*)&O.qstop[q]) st = 1;
                }
                stop = __shfl_sync(0xffffffffu, st, 0) != 0;
                if (stop) break;
            }
            const int64_t idx = sn + lane;
            bool ok = idx < ghi;
            uint32_t cnd = 0;
            if (ok) { cnd = __ldg(gen + idx); lb += 4; }
            if (lane == 0) fb += 4ull * (unsigned long long)(ghi - sn < 32 ? ghi - sn : 32);
            for (int x = 0; x <= ne; x++) {                     // the tree list, then the non-tree lists
                if (x == src) continue;
                if (!__any_sync(0xffffffffu, ok)) break;
                const uint32_t* L = x == 0 ? P.t_idx[d] : P.n_idx[e0 + x - 1];
                const int64_t lo = T.lo[x], hi = T.hi[x];
                uint32_t c = (uint32_t)cur[x];
                ok = warp_member(L + lo, (uint32_t)(hi - lo), &c, cnd, ok, &lb);
                __syncwarp();
                if (lane == 0) cur[x] = c;
                __syncwarp();
            }
            uint32_t sl = P.same_lab[d];
            if (sl) {
                const uint32_t pm = __ballot_sync(0xffffffffu, ok);
                if (lane == 0) fb += 4ull * __popc(pm);
                int32_t gc = -1;
                if (ok) { gc = __ldg(P.cand[d] + cnd); lb += 4; }
                while (sl) {
                    const int p = __ffs(sl) - 1;
                    sl &= sl - 1;
                    if (T.g[p] == gc) ok = false;
                }
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) local += __popc(mask);
        }
        if (lane == 0) flush_count(O, q, local);
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicExch(&ring->state[got % kRing], (uint32_t)(2 * (got / kRing) + 2));   // free for ticket + kRing
        }
    }
}

// BATCH: plans[q] per query (chunk flags carry q, nchunks is read from
// *nchunks_dev); otherwise the single plan P0 and the nchunks argument.
// WS: the warp-specialised variant (O.validators validator warps per CTA,
// the last warps; no counting pass, no embeddings written).
template <bool STATS, bool EMIT, bool BATCH, bool WS = false>
__global__ void __launch_bounds__(256, 4) k_match(const __grid_constant__ MatchPlan P0,
                                               const MatchPlan* __restrict__ plans,
                                               const Chunk* __restrict__ chunks, int64_t nchunks,
                                               const int64_t* __restrict__ nchunks_dev, MatchOut O) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (BATCH) nchunks = *nchunks_dev;
    const int warp_words = BATCH ? plans[0].warp_words : P0.warp_words;   // one stride for all queries
    uint32_t* sbuf = smem + (size_t)warp * warp_words;                   // [depth][32]
    uint32_t* sm = sbuf + kMaxK * 32;                                   // m[position]
    int32_t* sg = (int32_t*)(sm + kMaxK);                               // data vertex per position
    int32_t* gsrc = sg + kMaxK;                                          // per depth: generator list (as Chunk.pad)
    int64_t* tcur = (int64_t*)(gsrc + kMaxK);                            // per depth: tree-list cursor
    int64_t* ncur = tcur + kMaxK;                                        // per non-tree edge: list cursor
    unsigned long long iter = 0;
    const unsigned long long deadline = *O.deadline;
    unsigned long long lb = 0;             // this lane's bytes requested (entries of 4 B, offsets of 8 B)
    // lane 0: the floor of the bytes, what any search over the CST that scans
    // the shortest list into each position must read: per extension of a
    // partial result to position d, the new image (4 B), the offsets of the
    // tree list and of each earlier non-tree neighbour's list into d (16 B
    // each) and every entry of the generator list (4 B); per candidate that
    // passes the list checks while an earlier position has its label, its
    // data vertex (4 B); per embedding written, its row (4|V(q)| B).  A static
    // chunk that starts at position j > 0 counts its run's extension the same
    // way; a donated run counts only what it scans.
    unsigned long long fb = 0;
    unsigned long long local = 0;          // lane 0: count not yet flushed
    // warp-specialised: the ring after the warps' regions; expanders first
    VRing* ring = nullptr;
    const int nexp = WS ? (int)(blockDim.x >> 5) - O.validators : (int)(blockDim.x >> 5);
    if (WS) {
        ring = (VRing*)(smem + (((size_t)(blockDim.x >> 5) * warp_words + 3) & ~(size_t)3));
        if (threadIdx.x == 0) {
            ring->head = 0;
            ring->tail = 0;
            for (int i = 0; i < kRing; i++) ring->state[i] = 0;
            ring->active = nexp;
        }
        __syncthreads();
    }

    if (WS && warp >= nexp) {
        validate_tasks<BATCH>(P0, plans, ring, tcur, O, deadline, lb, fb);
    } else {
    for (;;) {
        unsigned long long ci = 0;
        int kind = 0;
        if (lane == 0) kind = acquire(O, nchunks, deadline, &ci);
        kind = __shfl_sync(0xffffffffu, kind, 0);
        ci = __shfl_sync(0xffffffffu, ci, 0);
        if (kind == 0) break;
        // the item's fields, read once.  A donated run was written by another
        // warp during this launch: read it from L2 (ld.global.cg), never from
        // an L1 line that may hold an older copy of its bytes.
        const Chunk* chp = kind == 1 ? chunks + ci : O.dq + ci % O.dq_cap;
        int j;
        uint32_t ch_a, ch_b, ch_pad, ch_pre;
        if (kind == 1) {
            j = chp->j; ch_a = chp->a; ch_b = chp->b; ch_pad = chp->pad;
            ch_pre = lane < j ? chp->prefix[lane] : 0u;
        } else {
            j = __ldcg(&chp->j); ch_a = __ldcg(&chp->a); ch_b = __ldcg(&chp->b); ch_pad = __ldcg(&chp->pad);
            ch_pre = lane < j ? __ldcg(&chp->prefix[lane]) : 0u;
            __syncwarp();
            if (lane == 0) {                      // hand the cell back for ticket ci + dq_cap
                __threadfence();
                atomicExch(&O.dq_state[ci % O.dq_cap], (uint32_t)(2 * (ci / O.dq_cap) + 2));
            }
        }
        const uint32_t q = BATCH ? (ch_pad >> 8) : 0u;
        const MatchPlan& P = BATCH ? plans[q] : P0;
        const int k = P.k;
        if (BATCH) {
            // this query already reached its limit?  One lane reads the flag and
            // broadcasts it: another warp may set it at any moment, and lanes
            // reading it separately could take different branches and then
            // never meet at the warp-wide operations that follow.
            int qs = 0;
            if (lane == 0) qs = *(volatile int*)&O.qstop[q];
            if (__shfl_sync(0xffffffffu, qs, 0)) {
                if (lane == 0) atomicAdd(O.outstanding, ~0ull);
                __syncwarp();
                continue;
            }
        }
        uint32_t m_reg = ch_pre;                               // lane p: candidate index of position p
        int32_t g_reg = -1;                                    // lane p: data vertex of position p
        if (lane < j) g_reg = P.cand[lane][m_reg];
        sm[lane] = m_reg;
        sg[lane] = g_reg;
        __syncwarp();
        // ---- the prefix must itself be a partial embedding (non-tree edges, injectivity)
        bool ok_prefix = true;
        if (lane < j) lb += 4 + 4;                              // prefix entry + its data vertex
        if (lane < j && lane > 0) {
            for (int e = P.nt_begin[lane]; e < P.nt_begin[lane + 1]; e++) {
                uint32_t mf = sm[P.nt_from[e]];
                int64_t lo = P.n_off[e][mf], hi = P.n_off[e][mf + 1];
                unsigned long long pr = 0;
                if (!bsearch_u32(P.n_idx[e], lo, hi, m_reg, &pr)) ok_prefix = false;
                lb += 16 + 4 * pr;
            }
            uint32_t sl = P.same_lab[lane];
            while (sl) {
                int p = __ffs(sl) - 1;
                sl &= sl - 1;
                if (sg[p] == g_reg) ok_prefix = false;
            }
        }
        unsigned long long ccount = 0;         // lane 0: this item's count
        if (__all_sync(0xffffffffu, ok_prefix)) {
            if (kind == 1 && j > 0 && lane == 0) fb += 4 + 16 + 16ull * (P.nt_begin[j + 1] - P.nt_begin[j]);
            // ---- depth j: the item's run of L_j
            int d = j;
            int64_t seg_next = 0, seg_end = 0, seg_base = 0;   // lane d: depth d's list scan
            uint32_t bcnt = 0, bcur = 0;                        // lane d: buffered survivors
            {
                // the run [a, b) is of the tree list of position j, or of a non-tree
                // list into j (a donated run of a depth that generated from it)
                const int src = run_source(ch_pad);
                int64_t base = 0;
                if (src == 0) {
                    if (j > 0) {
                        uint32_t mp = __shfl_sync(0xffffffffu, m_reg, P.par[j]);
                        base = P.t_off[j][mp];
                    }
                } else {
                    const int e = P.nt_begin[j] + src - 1;
                    uint32_t mf = __shfl_sync(0xffffffffu, m_reg, P.nt_from[e]);
                    base = P.n_off[e][mf];
                }
                int64_t lo = base + ch_a, hi = base + ch_b;
                if (lane == d) { seg_next = lo; seg_end = hi; seg_base = base; }
                if (lane == 0) {
                    gsrc[j] = src;
                    tcur[j] = 0;
                    lb += (j > 0 ? 16 : 0) + 16ull * (P.nt_begin[j + 1] - P.nt_begin[j]);
                }
                for (int e = P.nt_begin[j] + lane; e < P.nt_begin[j + 1]; e += 32) ncur[e] = 0;
                __syncwarp();
            }
            for (;;) {
                ++iter;
                if ((iter & 255) == 0) {
                    int stop = 0;
                    if (lane == 0) {
                        flush_count(O, q, local);
                        if (deadline && global_timer_ns() > deadline) atomicOr(O.status, kStatusTimeout);
                        stop = vload(O.status) & (kStatusTimeout | kStatusLimit);
                        if (BATCH && *(volatile int*)&O.qstop[q]) stop = 1;
                    }
                    if (__shfl_sync(0xffffffffu, stop, 0)) break;
                }
                if (O.dq_cap && (iter & 63) == 0) {
                    // give work away when some warp is idle
                    unsigned int idl = 0;
                    if (lane == 0) idl = *(volatile unsigned int*)O.idle;
                    idl = __shfl_sync(0xffffffffu, idl, 0);
                    if (idl) {
                        bool can = lane >= j && lane <= d && (seg_end - seg_next) >= 2;
                        uint32_t cm = __ballot_sync(0xffffffffu, can);
                        if (cm) {
                            int dd = __ffs(cm) - 1;
                            // claim the next ticket whose cell is free; a full
                            // ring (or a lost race, a few times) keeps the work here
                            unsigned long long slot = ~0ull;
                            if (lane == 0) {
                                unsigned long long t = vload(O.dq_tail);
                                for (int tries = 0; tries < 4; tries++) {
                                    uint32_t st = *(volatile uint32_t*)&O.dq_state[t % O.dq_cap];
                                    uint32_t g2 = (uint32_t)(2 * (t / O.dq_cap));
                                    if (st == g2) {
                                        unsigned long long prev = atomicCAS(O.dq_tail, t, t + 1);
                                        if (prev == t) { slot = t; break; }
                                        t = prev;
                                    } else if (st < g2) {
                                        break;                            // its previous run is not taken yet
                                    } else {
                                        t = vload(O.dq_tail);
                                    }
                                }
                            }
                            slot = __shfl_sync(0xffffffffu, slot, 0);
                            if (slot != ~0ull) {
                                int64_t sn_ = __shfl_sync(0xffffffffu, seg_next, dd);
                                int64_t se_ = __shfl_sync(0xffffffffu, seg_end, dd);
                                int64_t sb_ = __shfl_sync(0xffffffffu, seg_base, dd);
                                int64_t mid = sn_ + (se_ - sn_) / 2;
                                Chunk* dst = &O.dq[slot % O.dq_cap];
                                if (lane < kMaxK) dst->prefix[lane] = lane < dd ? sm[lane] : 0u;
                                if (lane == 0) {
                                    atomicAdd(O.outstanding, 1ull);
                                    dst->j = dd;
                                    dst->a = (uint32_t)(mid - sb_);
                                    dst->b = (uint32_t)(se_ - sb_);
                                    dst->pad = kDonated | ((uint32_t)gsrc[dd] << 1) | (q << 8);
                                    dst->w = 0;
                                    dst->id = 0;
                                }
                                __syncwarp();
                                if (lane == 0) {
                                    __threadfence();
                                    atomicExch(&O.dq_state[slot % O.dq_cap], (uint32_t)(2 * (slot / O.dq_cap) + 1));
                                }
                                if (lane == dd) seg_end = mid;
                            }
                        }
                    }
                }
                uint32_t cur_d = __shfl_sync(0xffffffffu, bcur, d);
                uint32_t cnt_d = __shfl_sync(0xffffffffu, bcnt, d);
                if (cur_d < cnt_d) {
                    // expand the next buffered survivor of depth d
                    uint32_t v = sbuf[d * 32 + cur_d];
                    if (lane == d) { bcur++; m_reg = v; g_reg = P.cand[d][v]; sm[d] = v; sg[d] = g_reg; lb += 4; }
                    d++;
                    uint32_t mp = __shfl_sync(0xffffffffu, m_reg, P.par[d]);
                    int64_t lo = P.t_off[d][mp], hi = P.t_off[d][mp + 1];
                    // Generator list: the candidates of depth d are the intersection of
                    // the tree list and every non-tree list into d, all sorted over
                    // C(u_d).  Scan the shortest (ties to the tree list, then to the
                    // earlier non-tree edge) and check the others: the same set.
                    int src = 0;
                    const int64_t tlo = lo, thi = hi;     // the tree list's range
                    const int e0 = P.nt_begin[d], ne = P.nt_begin[d + 1] - e0;
                    int64_t elo = 0, elen = 0;            // lane e < ne: non-tree edge e0 + e's range
                    if (ne > 0) {
                        uint32_t mf = __shfl_sync(0xffffffffu, m_reg, lane < ne ? P.nt_from[e0 + lane] : 0);
                        uint32_t key = 0xFFFFFFFFu;           // (length, lane), lists shorter than the tree list
                        if (lane < ne) {
                            elo = P.n_off[e0 + lane][mf];
                            elen = P.n_off[e0 + lane][mf + 1] - elo;
                            if (elen < hi - lo)
                                key = ((uint32_t)(elen < (1 << 26) ? elen : (1 << 26) - 1) << 5) | (uint32_t)lane;
                        }
                        uint32_t best = __reduce_min_sync(0xffffffffu, key);
                        if (best != 0xFFFFFFFFu) {
                            int bi = (int)(best & 31u);
                            src = bi + 1;
                            lo = __shfl_sync(0xffffffffu, elo, bi);
                            hi = lo + __shfl_sync(0xffffffffu, elen, bi);
                        }
                    }
                    if (WS && d == k - 1) {
                        // the last position: hand the extension to a validator warp
                        unsigned long long t = ~0ull;
                        if (lane == 0) t = ring_claim(ring);
                        t = __shfl_sync(0xffffffffu, t, 0);
                        if (t != ~0ull) {
                            VTask& T = ring->task[t % kRing];
                            if (lane == 0) { T.q = q; T.src = src; T.lo[0] = tlo; T.hi[0] = thi; }
                            if (lane < ne) { T.lo[1 + lane] = elo; T.hi[1 + lane] = elo + elen; }
                            if (lane < d) T.g[lane] = g_reg;
                            __threadfence_block();
                            __syncwarp();
                            if (lane == 0) {
                                atomicExch(&ring->state[t % kRing], (uint32_t)(2 * (t / kRing) + 1));
                                lb += 16 + 16ull * ne;
                                fb += 4 + 16 + 16ull * ne;
                            }
                            d--;
                            continue;
                        }
                        // a full ring: this warp scans the extension itself
                    }
                    if (lane == d) { seg_next = lo; seg_end = hi; seg_base = lo; bcnt = 0; bcur = 0; }
                    if (lane == 0) {
                        gsrc[d] = src;
                        tcur[d] = 0;
                        lb += 16 + 16ull * (P.nt_begin[d + 1] - P.nt_begin[d]);
                        fb += 4 + 16 + 16ull * (P.nt_begin[d + 1] - P.nt_begin[d]);
                    }
                    for (int e = P.nt_begin[d] + lane; e < P.nt_begin[d + 1]; e += 32) ncur[e] = 0;
                    __syncwarp();
                    continue;
                }
                int64_t sn = __shfl_sync(0xffffffffu, seg_next, d);
                int64_t se = __shfl_sync(0xffffffffu, seg_end, d);
                if (!EMIT && d == k - 1 && d > 0 && sn < se) {
                    // The last position: its segments one after another in a
                    // loop of their own, the same Generator, EdgeValidator and
                    // VisitedValidator steps as below, with each list's first
                    // entry, length and merge cursor held by one lane (lane 0
                    // the tree list, lane x the x-th non-tree list into d).
                    // Back to the main loop when the run ends and before every
                    // 64th step, where the periodic checks and donations are.
                    const int src = gsrc[d];
                    const int e0 = P.nt_begin[d], ne = P.nt_begin[d + 1] - e0;
                    const int from = lane == 0 ? P.par[d] : (lane <= ne ? P.nt_from[e0 + lane - 1] : 0);
                    const uint32_t mf = __shfl_sync(0xffffffffu, m_reg, from);
                    const uint32_t* lp = nullptr;
                    uint32_t ln = 0, lc = 0;
                    if (lane <= ne) {
                        const int64_t* off = lane == 0 ? P.t_off[d] : P.n_off[e0 + lane - 1];
                        const int64_t lo = off[mf];
                        lp = (lane == 0 ? P.t_idx[d] : P.n_idx[e0 + lane - 1]) + lo;
                        ln = (uint32_t)(off[mf + 1] - lo);
                        lc = (uint32_t)(lane == 0 ? tcur[d] : ncur[e0 + lane - 1]);
                    }
                    const uint32_t* gp = (const uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)lp, src);
                    const int64_t sb = __shfl_sync(0xffffffffu, seg_base, d);
                    uint32_t r = (uint32_t)(sn - sb);
                    const uint32_t re = (uint32_t)(se - sb);
                    const uint32_t sl0 = P.same_lab[d];
                    const int32_t* cd = P.cand[d];
                    for (;;) {
                        const uint32_t i = r + lane;
                        bool ok = i < re;
                        uint32_t cnd = 0;
                        if (ok) { cnd = __ldg(gp + i); lb += 4; }
                        if (lane == 0) fb += 4ull * (re - r < 32 ? re - r : 32);
                        for (int x = 0; x <= ne; x++) {
                            if (x == src) continue;
                            if (!__any_sync(0xffffffffu, ok)) break;
                            const uint32_t* L = (const uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)lp, x);
                            const uint32_t n = __shfl_sync(0xffffffffu, ln, x);
                            uint32_t c = __shfl_sync(0xffffffffu, lc, x);
                            ok = warp_member(L, n, &c, cnd, ok, &lb);
                            if (lane == x) lc = c;
                        }
                        if (sl0) {
                            const uint32_t pm = __ballot_sync(0xffffffffu, ok);
                            if (lane == 0) fb += 4ull * __popc(pm);
                            int32_t gc = -1;
                            if (ok) { gc = __ldg(cd + cnd); lb += 4; }
                            uint32_t sl = sl0;
                            while (sl) {
                                const int p = __ffs(sl) - 1;
                                sl &= sl - 1;
                                if (__shfl_sync(0xffffffffu, g_reg, p) == gc) ok = false;
                            }
                        }
                        const uint32_t mask = __ballot_sync(0xffffffffu, ok);
                        if (STATS && lane == 0) atomicAdd(&O.stats[d], (unsigned long long)__popc(mask));
                        if (lane == 0) { local += __popc(mask); ccount += __popc(mask); }
                        r += 32;
                        if (r >= re || ((iter + 1) & 63) == 0) break;
                        ++iter;
                    }
                    if (lane == d) seg_next = sb + r;
                    if (lane == 0) tcur[d] = lc;
                    else if (lane <= ne) ncur[e0 + lane - 1] = lc;
                    __syncwarp();
                    continue;
                }
                if (sn < se) {
                    // Generator: next 32 entries of depth d's list
                    int64_t idx = sn + lane;
                    bool ok = idx < se;
                    uint32_t cnd = 0;
                    const int src = gsrc[d];
                    const int gen_e = P.nt_begin[d] + src - 1;          // the generating non-tree edge (src > 0)
                    if (ok) {
                        cnd = (d == 0) ? (uint32_t)idx : __ldg((src == 0 ? P.t_idx[d] : P.n_idx[gen_e]) + idx);
                        if (d > 0) lb += 4;
                    }
                    if (d > 0 && lane == 0) fb += 4ull * (unsigned long long)(se - sn < 32 ? se - sn : 32);
                    // a non-tree list generates: the tree list is checked like the others
                    if (src != 0 && __any_sync(0xffffffffu, ok)) {
                        uint32_t mp = __shfl_sync(0xffffffffu, m_reg, P.par[d]);
                        int64_t lo = P.t_off[d][mp], hi = P.t_off[d][mp + 1];
                        uint32_t cur = (uint32_t)tcur[d];
                        ok = warp_member(P.t_idx[d] + lo, (uint32_t)(hi - lo), &cur, cnd, ok, &lb);
                        __syncwarp();
                        if (lane == 0) tcur[d] = cur;
                        __syncwarp();
                    }
                    // EdgeValidator (most selective edge first; stop once no lane is pending)
                    for (int e = P.nt_begin[d]; e < P.nt_begin[d + 1]; e++) {
                        if (e == gen_e) continue;
                        if (!__any_sync(0xffffffffu, ok)) break;
                        uint32_t mf = __shfl_sync(0xffffffffu, m_reg, P.nt_from[e]);
                        int64_t lo = P.n_off[e][mf], hi = P.n_off[e][mf + 1];
                        uint32_t cur = (uint32_t)ncur[e];
                        ok = warp_member(P.n_idx[e] + lo, (uint32_t)(hi - lo), &cur, cnd, ok, &lb);
                        __syncwarp();
                        if (lane == 0) ncur[e] = cur;
                        __syncwarp();
                    }
                    // VisitedValidator
                    int32_t gc = -1;
                    uint32_t sl = P.same_lab[d];
                    if (sl || (EMIT && d == k - 1)) {
                        if (sl) {
                            const uint32_t pm = __ballot_sync(0xffffffffu, ok);
                            if (lane == 0) fb += 4ull * __popc(pm);
                        }
                        if (ok) { gc = __ldg(P.cand[d] + cnd); lb += 4; }
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
                    if (STATS && lane == 0) atomicAdd(&O.stats[d], (unsigned long long)__popc(mask));
                    if (d == k - 1) {
                        if (lane == 0) { local += __popc(mask); ccount += __popc(mask); }
                        if (EMIT && !BATCH && mask) {
                            unsigned long long base = 0;
                            if (lane == 0) base = atomicAdd(O.emb_slot, (unsigned long long)__popc(mask));
                            base = __shfl_sync(0xffffffffu, base, 0);
                            unsigned long long slot = base + __popc(mask & lanemask_lt());
                            if (lane == 0 && base < O.emb_cap) {
                                const unsigned long long nw = __popc(mask);
                                fb += 4ull * k * (nw < O.emb_cap - base ? nw : O.emb_cap - base);
                            }
                            bool wr = ok && slot < O.emb_cap;
                            if (wr) lb += 4ull * k;
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
            flush_count(O, q, local);
            if (O.chunk_counts && kind == 1) O.chunk_counts[ci] = ccount;
            atomicAdd(O.outstanding, ~0ull);   // -1
        }
        __syncwarp();
    }
    if (WS && lane == 0) {                     // this expander's tasks are all published
        __threadfence_block();
        atomicSub(&ring->active, 1);
    }
    }
    for (int o = 16; o > 0; o >>= 1) lb += __shfl_xor_sync(0xffffffffu, lb, o);
    if (lane == 0 && lb) atomicAdd(O.bytes, lb);
    if (lane == 0 && fb) atomicAdd(O.floor, fb);
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
    // Non-tree edges into each position, the shortest lists on average (the
    // likeliest to reject a candidate) first: a segment stops checking once
    // no candidate is left.  The order does not change the result.
    int e = 0;
    for (int i = 0; i < k; i++) {
        P.nt_begin[i] = e;
        int ts[kMaxNT], nts = 0;
        for (int t = 0; t < c->nnt; t++)
            if (c->pos[c->nt_to[t]] == i) ts[nts++] = t;
        auto avg = [&](int t) {
            int64_t rows = c->ncand[c->nt_from[t]];
            return (double)c->n_entries[t] / (double)(rows > 0 ? rows : 1);
        };
        std::stable_sort(ts, ts + nts, [&](int a, int b) { return avg(a) < avg(b); });
        for (int x = 0; x < nts; x++) {
            int t = ts[x];
            P.nt_from[e] = c->pos[c->nt_from[t]];
            P.n_off[e] = c->n_off[t];
            P.n_idx[e] = c->n_idx[t];
            e++;
        }
    }
    P.nt_begin[k] = e;
    P.warp_words = kWarpBaseWords + 2 * e;
    return P;
}

size_t smem_bytes(const MatchPlan& P, int warps) { return (size_t)warps * P.warp_words * sizeof(uint32_t); }

// the warp-specialised variant: its validator warps per CTA (0: the fused kernel)
int ws_validators(const fast_config& cfg, int warps) {
    if (cfg.matcher_rule != 1 || warps < 2) return 0;
    return cfg.validators > 0 ? std::min(cfg.validators, warps - 1) : warps / 2;
}

// dynamic shared memory of a launch: the warps' regions, then (warp-
// specialised) the task ring on a 16-byte boundary
size_t launch_smem(int warps, int warp_words, bool ws) {
    const size_t words = ((size_t)warps * warp_words + 3) & ~(size_t)3;
    return words * sizeof(uint32_t) + (ws ? sizeof(VRing) : 0);
}

// Opt every matcher variant in to the largest dynamic shared memory any
// query can ask for (8 warps of a 32-vertex query with all its non-tree
// cursors), once per device.  The attribute is process-wide: setting it per
// launch to that launch's size would let a concurrent caller on another
// thread lower it between someone else's set and launch.
constexpr size_t kMatcherSmemMax = (size_t)8 * (kWarpBaseWords + 2 * kMaxNT) * sizeof(uint32_t) + 16 + sizeof(VRing);

int matcher_smem_optin(size_t bytes) {
    if (bytes > kMatcherSmemMax) return set_error(FAST_ERR_INVALID, "matcher: %zu bytes of shared memory per CTA", bytes);
    static std::mutex mu;
    static uint64_t done = 0;                  // bit per device
    int dev = 0;
    FAST_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && (done >> dev) & 1) return FAST_OK;
    const int sz = (int)kMatcherSmemMax;
    FAST_CUDA(cudaFuncSetAttribute(k_match<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    FAST_CUDA(cudaFuncSetAttribute(k_match<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    FAST_CUDA(cudaFuncSetAttribute(k_match<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    FAST_CUDA(cudaFuncSetAttribute(k_match<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    FAST_CUDA(cudaFuncSetAttribute(k_match<false, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    FAST_CUDA(cudaFuncSetAttribute(k_match<false, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz));
    if (dev < 64) done |= 1ull << dev;
    return FAST_OK;
}

// counter block layout (unsigned long long words)
enum { kNext = 0, kTotal, kSlot, kStatus, kBytes, kFloor, kHead, kTail, kOut, kIdle, kDeadline, kQStop, kStats,
       kCtrWords = kStats + kMaxK + 1 };
constexpr uint64_t kQueueCap = 1 << 16;

// cells of the donation ring for a launch: cfg.queue_cells, at most (and by default) cap
uint64_t ring_cells(const fast_config& cfg, uint64_t cap) {
    return cfg.queue_cells > 0 ? std::min<uint64_t>((uint64_t)cfg.queue_cells, cap) : cap;
}

int run_match(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg_in, uint64_t kemb, uint32_t* emb_out,
              uint64_t* count_out, uint64_t* written_out, uint64_t* chunk_counts, uint64_t* stats_out,
              cudaStream_t s) {
    if (!c) return set_error(FAST_ERR_INVALID, "fast_match: cst is NULL");
    if (kemb > 0 && !emb_out) return set_error(FAST_ERR_INVALID, "fast_match: k > 0 needs emb_out");
    if (chunks && chunks->c != c) return set_error(FAST_ERR_INVALID, "fast_match: chunks belong to another CST");
    PoolScope scratch(s);                        // counters, donation ring, staging: temporaries
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
    // per-chunk counts and the counting pass need every run done where it was
    // scheduled (a donated run re-reads its prefix), so they run without donation
    const bool donate = chunk_counts == nullptr && stats_out == nullptr;
    unsigned long long* ctr = nullptr;
    Chunk* dq = nullptr;
    uint32_t* dq_state = nullptr;
    const uint64_t cells = ring_cells(cfg, kQueueCap);
    rc = dalloc(&ctr, kCtrWords, s);
    if (rc == FAST_OK && donate) rc = dalloc(&dq, cells, s);
    if (rc == FAST_OK && donate) rc = dalloc(&dq_state, cells, s);
    uint32_t* emb_dev = emb_out;
    uint32_t* staged = nullptr;
    bool timed = false;
    uint64_t emb_cap = kemb;
    if (cfg.limit > 0 && cfg.limit < emb_cap) emb_cap = cfg.limit;
    if (rc == FAST_OK && kemb > 0) {
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, emb_out);
        cudaGetLastError();
        bool device_ok = e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        if (!device_ok) {
            rc = dalloc(&staged, emb_cap * (uint64_t)c->k, s);
            emb_dev = staged;
        }
    }
    if (rc == FAST_OK) {
        cudaMemsetAsync(ctr, 0, kCtrWords * sizeof(unsigned long long), s);
        unsigned long long out0 = (unsigned long long)nchunks;
        cudaMemcpyAsync(ctr + kOut, &out0, sizeof(out0), cudaMemcpyHostToDevice, s);
        if (donate) cudaMemsetAsync(dq_state, 0, cells * sizeof(uint32_t), s);
        MatchOut O;
        O.next_chunk = ctr + kNext; O.total = ctr + kTotal; O.emb_slot = ctr + kSlot; O.status = (int*)(ctr + kStatus);
        O.qstop = (int*)(ctr + kQStop); O.nq = 1;
        // without a partition the root runs are internal: the whole CST is the one chunk
        O.chunk_counts = chunks ? chunk_counts : nullptr; O.emb = emb_dev; O.emb_cap = emb_cap;
        O.stats = stats_out ? ctr + kStats : nullptr;
        O.bytes = ctr + kBytes;
        O.floor = ctr + kFloor;
        O.deadline = ctr + kDeadline;
        O.limit = cfg.limit;
        O.dq = dq; O.dq_state = dq_state; O.dq_cap = donate ? cells : 0;
        O.dq_head = ctr + kHead; O.dq_tail = ctr + kTail; O.outstanding = ctr + kOut;
        O.idle = (unsigned int*)(ctr + kIdle);
        // the warp-specialised kernel for counting launches that ask for it
        const int nval = (!stats_out && kemb == 0 && chunk_counts == nullptr) ? ws_validators(cfg, warps) : 0;
        O.validators = nval;
        unsigned long long budget_ns = cfg.time_budget_s > 0 ? (unsigned long long)(cfg.time_budget_s * 1e9) : 0ull;
        if (budget_ns) { k_set_deadline<<<1, 1, 0, s>>>(ctr + kDeadline, budget_ns); note_launch(); }
        if (nchunks > 0) {
            int64_t grid = (int64_t)num_sms() * bps;
            if (!donate) grid = std::max<int64_t>(1, std::min<int64_t>(grid, ceil_div(nchunks, warps)));
            size_t sh = launch_smem(warps, P.warp_words, nval > 0);
            rc = matcher_smem_optin(sh);
            if (rc == FAST_OK) {
                EventPair& ev = match_events();
                if (ev.ok) cudaEventRecord(ev.a, s);
                if (stats_out) { k_match<true, false, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O); note_launch(); }
                else if (kemb > 0) { k_match<false, true, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O); note_launch(); }
                else if (nval > 0) { k_match<false, false, false, true><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O); note_launch(); }
                else { k_match<false, false, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O); note_launch(); }
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) rc = cuda_status(e, "matcher launch", __FILE__, __LINE__);
                if (ev.ok) cudaEventRecord(ev.b, s);
                timed = ev.ok;
            }
        }
    }
    unsigned long long h[kCtrWords];
    memset(h, 0, sizeof(h));
    if (rc == FAST_OK && !chunks && chunk_counts) {
        cudaError_t e = cudaMemcpyAsync(chunk_counts, ctr + kTotal, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_match chunk count", __FILE__, __LINE__);
    }
    if (rc == FAST_OK) {
        cudaError_t e = cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_match", __FILE__, __LINE__);
        g_last_match_ms = 0.0;
        g_last_match_bytes = h[kBytes];
        g_last_match_floor = h[kFloor];
        if (rc == FAST_OK && timed) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, match_events().a, match_events().b) == cudaSuccess) g_last_match_ms = ms;
            else cudaGetLastError();
        }
    }
    uint64_t written = std::min<uint64_t>(emb_cap, h[kSlot]);
    if (rc == FAST_OK && staged) {
        cudaError_t e = written ? cudaMemcpyAsync(emb_out, staged, written * c->k * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "fast_match embedding readback", __FILE__, __LINE__);
    }
    dfree(ctr, s); dfree(own, s); dfree(staged, s); dfree(dq, s); dfree(dq_state, s);
    if (rc != FAST_OK) return rc;
    uint64_t total = h[kTotal];
    if (cfg.limit > 0 && total > cfg.limit) total = cfg.limit;
    if (count_out) *count_out = total;
    if (written_out) *written_out = written;
    if (stats_out) {
        stats_out[0] = h[kBytes];
        for (int i = 0; i < c->k; i++) stats_out[1 + i] = h[kStats + i];
    }
    int st = (int)h[kStatus];
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

extern "C" uint64_t fast_last_match_bytes(void) { return g_last_match_bytes; }

extern "C" uint64_t fast_last_match_floor_bytes(void) { return g_last_match_floor; }

// ------------------------------------------------------ allocation-free matcher
//
// Scratch of fast_match_noalloc, in one file-scope device array: the counter
// block, the queue of donated runs with its ready flags, and the run
// descriptors used when no partition is given.  Host code must not pass the
// symbol itself to a kernel (on the host it only names a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.

namespace {

constexpr int kNoAllocQueue = 4096;                   // donated runs
constexpr int kNoAllocRuns = 32768;                   // root runs when chunks == NULL
constexpr size_t kNaCtrBytes = ((kCtrWords * sizeof(unsigned long long) + 255) / 256) * 256;
constexpr size_t kNaQueueBytes = kNoAllocQueue * sizeof(Chunk);
constexpr size_t kNaReadyBytes = ((kNoAllocQueue * sizeof(uint32_t) + 255) / 256) * 256;
constexpr size_t kNaRunsBytes = kNoAllocRuns * sizeof(Chunk);
constexpr size_t kNoAllocBytes = kNaCtrBytes + kNaQueueBytes + kNaReadyBytes + kNaRunsBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int noalloc_scratch(unsigned char** out) {
    int dev = 0;
    FAST_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FAST_ERR_INVALID, "fast_match_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        unsigned char* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FAST_OK;
}

__global__ void k_root_runs(Chunk* runs, uint64_t parts, uint64_t nr) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= parts) return;
    Chunk c;
    memset(&c, 0, sizeof(c));
    c.j = 0;
    c.a = (uint32_t)(i * nr / parts);
    c.b = (uint32_t)((i + 1) * nr / parts);
    runs[i] = c;
}

int run_match_noalloc(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg_in, uint64_t kemb,
                      uint32_t* emb_out, uint64_t* count_out, uint64_t* written_out, cudaStream_t s) {
    if (!c) return set_error(FAST_ERR_INVALID, "fast_match_noalloc: cst is NULL");
    if (kemb > 0 && !emb_out) return set_error(FAST_ERR_INVALID, "fast_match_noalloc: k > 0 needs emb_out");
    if (chunks && chunks->c != c) return set_error(FAST_ERR_INVALID, "fast_match_noalloc: chunks belong to another CST");
    if (kemb > 0) {
        cudaPointerAttributes at;
        cudaError_t e = cudaPointerGetAttributes(&at, emb_out);
        cudaGetLastError();
        if (e != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged))
            return set_error(FAST_ERR_INVALID, "fast_match_noalloc: emb_out must be device memory (a host buffer would need a staging allocation)");
    }
    fast_config cfg = cfg_in ? *cfg_in : c->cfg;
    int warps = cfg.warps_per_block > 0 ? cfg.warps_per_block : 8;
    if (warps > 8) warps = 8;
    int bps = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : 4;
    unsigned char* base = nullptr;
    FAST_TRY(noalloc_scratch(&base));
    unsigned long long* ctr = (unsigned long long*)base;
    Chunk* dq = (Chunk*)(base + kNaCtrBytes);
    uint32_t* dq_state = (uint32_t*)(base + kNaCtrBytes + kNaQueueBytes);
    const uint64_t cells = ring_cells(cfg, kNoAllocQueue);
    Chunk* runs = (Chunk*)(base + kNaCtrBytes + kNaQueueBytes + kNaReadyBytes);
    const Chunk* dchunks = nullptr;
    int64_t nchunks = 0;
    if (chunks) { dchunks = chunks->d; nchunks = chunks->n; }
    else if (c->ncand[c->root] > 0) {
        uint64_t nr = (uint64_t)c->ncand[c->root];
        uint64_t want = (uint64_t)num_sms() * bps * warps * 4;
        uint64_t parts = std::min<uint64_t>(nr, want);
        if (parts > (uint64_t)kNoAllocRuns)
            return set_error(FAST_ERR_INVALID,
                             "fast_match_noalloc: %llu root runs needed, the static scratch holds %d "
                             "(pass a partition or fewer warps per SM)", (unsigned long long)parts, kNoAllocRuns);
        k_root_runs<<<(unsigned)ceil_div((int64_t)parts, 256), 256, 0, s>>>(runs, parts, nr);
        note_launch();
        dchunks = runs;
        nchunks = (int64_t)parts;
    }
    uint64_t emb_cap = kemb;
    if (cfg.limit > 0 && cfg.limit < emb_cap) emb_cap = cfg.limit;
    FAST_CUDA(cudaMemsetAsync(ctr, 0, kCtrWords * sizeof(unsigned long long), s));
    unsigned long long out0 = (unsigned long long)nchunks;
    FAST_CUDA(cudaMemcpyAsync(ctr + kOut, &out0, sizeof(out0), cudaMemcpyHostToDevice, s));
    FAST_CUDA(cudaMemsetAsync(dq_state, 0, cells * sizeof(uint32_t), s));
    MatchPlan P = make_plan(c);
    MatchOut O;
    O.next_chunk = ctr + kNext; O.total = ctr + kTotal; O.emb_slot = ctr + kSlot; O.status = (int*)(ctr + kStatus);
        O.qstop = (int*)(ctr + kQStop); O.nq = 1;
    O.chunk_counts = nullptr; O.emb = emb_out; O.emb_cap = emb_cap;
    O.stats = nullptr;
    O.bytes = ctr + kBytes;
    O.floor = ctr + kFloor;
    O.deadline = ctr + kDeadline;
    O.limit = cfg.limit;
    O.dq = dq; O.dq_state = dq_state; O.dq_cap = cells;
    O.dq_head = ctr + kHead; O.dq_tail = ctr + kTail; O.outstanding = ctr + kOut;
    O.idle = (unsigned int*)(ctr + kIdle);
    O.validators = 0;                                  // the fused kernel
    unsigned long long budget_ns = cfg.time_budget_s > 0 ? (unsigned long long)(cfg.time_budget_s * 1e9) : 0ull;
    if (budget_ns) { k_set_deadline<<<1, 1, 0, s>>>(ctr + kDeadline, budget_ns); note_launch(); }
    if (nchunks > 0) {
        int64_t grid = (int64_t)num_sms() * bps;
        size_t sh = smem_bytes(P, warps);
        FAST_TRY(matcher_smem_optin(sh));
        if (kemb > 0) k_match<false, true, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O);
        else k_match<false, false, false><<<(unsigned)grid, warps * 32, sh, s>>>(P, nullptr, dchunks, nchunks, nullptr, O);
        note_launch();
        FAST_CUDA(cudaGetLastError());
    }
    unsigned long long h[kCtrWords];
    FAST_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
    FAST_CUDA(cudaStreamSynchronize(s));
    uint64_t total = h[kTotal];
    if (cfg.limit > 0 && total > cfg.limit) total = cfg.limit;
    if (count_out) *count_out = total;
    if (written_out) *written_out = std::min<uint64_t>(emb_cap, h[kSlot]);
    int st = (int)h[kStatus];
    if (st & kStatusTimeout) return set_error(FAST_ERR_TIMEOUT, "fast_match_noalloc: time budget of %.3f s spent", cfg.time_budget_s);
    if (st & kStatusOverflow) return set_error(FAST_ERR_OVERFLOW, "fast_match_noalloc: count reached 2^64");
    return FAST_OK;
}

}  // namespace

extern "C" int fast_match_noalloc(const fast_cst* c, const fast_chunks* chunks, const fast_config* cfg, uint64_t k,
                                  uint32_t* emb_out, uint64_t* count_out, uint64_t* written_out, void* stream) {
    return run_match_noalloc(c, chunks, cfg, k, emb_out, count_out, written_out, (cudaStream_t)stream);
}

extern "C" uint64_t fast_match_noalloc_scratch_bytes(void) { return (uint64_t)kNoAllocBytes; }

// --------------------------------------------------- interface for batch.cu

namespace fast {

size_t match_plan_bytes() { return sizeof(MatchPlan); }

int match_plan_fill(const fast_cst* c, void* host_plan) {
    MatchPlan P = make_plan(c);
    memcpy(host_plan, &P, sizeof(P));
    return P.warp_words;
}

void match_plan_set_stride(void* host_plans, int nq, int warp_words) {
    MatchPlan* P = (MatchPlan*)host_plans;
    for (int i = 0; i < nq; i++) P[i].warp_words = warp_words;
}

size_t match_counter_words() { return kCtrWords; }
size_t match_chunk_bytes() { return sizeof(Chunk); }

// Enqueue one batched matcher launch (capturable: memsets and kernels only).
int match_batched_enqueue(const void* d_plans, int warp_words, const void* d_chunks, const int64_t* d_nchunks,
                          int max_q, unsigned long long* d_qtotal, int* d_qstop, unsigned long long* d_ctr,
                          void* d_dq, uint32_t* d_dq_state, uint64_t dq_cap, uint64_t limit, double budget_s,
                          int warps, int bps, int validators, cudaStream_t s) {
    MatchPlan dummy;
    memset(&dummy, 0, sizeof(dummy));
    dummy.warp_words = warp_words;
    const int nval = validators > 0 && warps >= 2 ? std::min(validators, warps - 1) : 0;
    size_t sh = launch_smem(warps, warp_words, nval > 0);
    FAST_CUDA(cudaMemsetAsync(d_ctr, 0, kCtrWords * sizeof(unsigned long long), s));
    FAST_CUDA(cudaMemsetAsync(d_qtotal, 0, (size_t)max_q * sizeof(unsigned long long), s));
    FAST_CUDA(cudaMemsetAsync(d_qstop, 0, (size_t)max_q * sizeof(int), s));
    FAST_CUDA(cudaMemsetAsync(d_dq_state, 0, dq_cap * sizeof(uint32_t), s));
    MatchOut O;
    memset(&O, 0, sizeof(O));
    O.next_chunk = d_ctr + kNext; O.total = d_qtotal; O.qstop = d_qstop; O.nq = max_q;
    O.emb_slot = d_ctr + kSlot; O.status = (int*)(d_ctr + kStatus);
    O.chunk_counts = nullptr; O.emb = nullptr; O.emb_cap = 0; O.stats = nullptr;
    O.bytes = d_ctr + kBytes; O.floor = d_ctr + kFloor; O.deadline = d_ctr + kDeadline; O.limit = limit;
    O.dq = (Chunk*)d_dq; O.dq_state = d_dq_state; O.dq_cap = dq_cap;
    O.dq_head = d_ctr + kHead; O.dq_tail = d_ctr + kTail; O.outstanding = d_ctr + kOut;
    O.idle = (unsigned int*)(d_ctr + kIdle);
    O.validators = nval;
    // outstanding = number of chunks, read on the device from *d_nchunks
    k_copy_word<<<1, 1, 0, s>>>(d_ctr + kOut, d_nchunks);
    note_launch();
    unsigned long long budget_ns = budget_s > 0 ? (unsigned long long)(budget_s * 1e9) : 0ull;
    if (budget_ns) { k_set_deadline<<<1, 1, 0, s>>>(d_ctr + kDeadline, budget_ns); note_launch(); }
    int64_t grid = (int64_t)num_sms() * bps;
    if (nval > 0)
        k_match<false, false, true, true><<<(unsigned)grid, warps * 32, sh, s>>>(dummy, (const MatchPlan*)d_plans,
                                                                                 (const Chunk*)d_chunks, 0, d_nchunks, O);
    else
        k_match<false, false, true><<<(unsigned)grid, warps * 32, sh, s>>>(dummy, (const MatchPlan*)d_plans,
                                                                           (const Chunk*)d_chunks, 0, d_nchunks, O);
    note_launch();
    FAST_CUDA(cudaGetLastError());
    return FAST_OK;
}

int match_smem_optin(size_t bytes) { return matcher_smem_optin(bytes); }

int match_status_of(const unsigned long long* h_ctr, uint64_t* bytes, uint64_t* floor) {
    if (bytes) *bytes = h_ctr[kBytes];
    if (floor) *floor = h_ctr[kFloor];
    return (int)h_ctr[kStatus];
}

}  // namespace fast
