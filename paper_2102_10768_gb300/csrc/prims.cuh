// Device-wide building blocks written for this library: exclusive scan,
// ordered predicate compaction over an index space (single pass, decoupled
// look-back; a two-pass form where the output size is needed first), and a
// stable LSD radix sort of 64-bit keys.  All are stream-ordered and take
// their scratch through dalloc on the caller's stream.
#pragma once

#include <algorithm>
#include <type_traits>
#include <utility>

#include "common.cuh"

namespace fast {

constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// Block-wide exclusive scan of ITEMS values per thread (blocked layout:
// thread t holds tile positions t*ITEMS .. t*ITEMS+ITEMS-1).  Returns the
// block total.  `warp_tmp` needs BLOCK/32 entries of shared memory.
template <class T, int BLOCK, int ITEMS>
__device__ __forceinline__ T block_exclusive_scan(T (&v)[ITEMS], T* warp_tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T local = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) { T x = v[i]; v[i] = local; local += x; }
    T incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = BLOCK / 32;
        T x = lane < NW ? warp_tmp[lane] : T(0);
        T y = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, y, off);
            if (lane >= off) y += t;
        }
        if (lane < NW) warp_tmp[lane] = y - x;       // exclusive
        if (lane == NW - 1) warp_tmp[NW] = y;         // total
    }
    __syncthreads();
    T base = warp_tmp[warp] + (incl - local);
#pragma unroll
    for (int i = 0; i < ITEMS; i++) v[i] += base;
    T total = warp_tmp[BLOCK / 32];
    __syncthreads();
    return total;
}

template <class T>
__global__ void k_scan_partials(const T* __restrict__ in, int64_t n, T* __restrict__ partials) {
    __shared__ T tmp[kScanBlock / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) v[i] = (base + i < n) ? in[base + i] : T(0);
    T tot = block_exclusive_scan<T, kScanBlock, kScanItems>(v, tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_apply(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                             const T* __restrict__ partials, T* __restrict__ total) {
    __shared__ T tmp[kScanBlock / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) v[i] = (base + i < n) ? in[base + i] : T(0);
    T tot = block_exclusive_scan<T, kScanBlock, kScanItems>(v, tmp);
    T off = partials ? partials[blockIdx.x] : T(0);
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) out[base + i] = v[i] + off;
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + tot;
}

// out[i] = in[0] + ... + in[i-1]; *total (device, nullable) = sum of all.
// in and out may alias.
template <class T>
int scan_exclusive(const T* in, T* out, int64_t n, T* total, cudaStream_t s) {
    if (n <= 0) {
        if (total) FAST_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return FAST_OK;
    }
    int64_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_apply<T><<<1, kScanBlock, 0, s>>>(in, out, n, (const T*)nullptr, total);
        note_launch();
        FAST_CUDA(cudaGetLastError());
        return FAST_OK;
    }
    T* part = nullptr;
    FAST_TRY(dalloc(&part, nb, s));
    k_scan_partials<T><<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, part);
    note_launch();
    int rc = cudaGetLastError() == cudaSuccess ? FAST_OK : set_error(FAST_ERR_CUDA, "scan partials launch");
    if (rc == FAST_OK) rc = scan_exclusive<T>(part, part, nb, (T*)nullptr, s);
    if (rc == FAST_OK) {
        k_scan_apply<T><<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, part, total);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "scan apply launch");
    }
    dfree(part, s);
    return rc;
}

// ---------------------------------------------------------------- compaction
//
// Ordered compaction over indices [0, n): F::eval(i, val) says whether index
// i is kept and what to write; kept values land in out[] in index order.
// F::begin(i0) is called once per thread before it evaluates indices i0,
// i0+1, ... in increasing order.  In the write pass F::tag(i), called right
// after eval(i), may return a non-negative tag (e.g. the row that index i
// starts); F::at(tag, rank) then receives the number of kept indices before
// i (used to write list offsets).

constexpr int kCompBlock = 128;
constexpr int kCompBlocksPerSM = 8;            // small blocks: one waiting on its look-back leaves 7 running
constexpr int kCompItems = 16;               // single-pass compaction: indices per thread
constexpr int kCompTile = kCompBlock * kCompItems;
constexpr int kEvalN = 8;                    // indices a functor's eval_n takes at once
static_assert(kCompItems % kEvalN == 0 && kCompItems <= 32, "a thread's kept indices form one 32-bit mask");
constexpr int kComp2Items = 8;               // the two-pass form (compact_alloc)
constexpr int kComp2Tile = kCompBlock * kComp2Items;

// A functor with a member `bool counting` has it set in the count pass, so
// that side effects of eval (marking a bitmap) happen once, in the write pass.
template <class F, class = void>
struct has_counting : std::false_type {};
template <class F>
struct has_counting<F, std::void_t<decltype(std::declval<F&>().counting)>> : std::true_type {};

template <class F>
__global__ void k_compact_count(F f, int64_t n, int64_t* __restrict__ counts) {
    __shared__ int64_t tmp[kCompBlock / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kComp2Tile + (int64_t)threadIdx.x * kComp2Items;
    int64_t v[kComp2Items];
    F g = f;
    if constexpr (has_counting<F>::value) g.counting = true;
    g.begin(base);
#pragma unroll
    for (int i = 0; i < kComp2Items; i++) {
        typename F::value_type x;
        v[i] = (base + i < n && g.eval(base + i, x)) ? 1 : 0;
    }
    int64_t tot = block_exclusive_scan<int64_t, kCompBlock, kComp2Items>(v, tmp);
    if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

template <class F>
__global__ void k_compact_write(F f, int64_t n, const int64_t* __restrict__ offs,
                                typename F::value_type* __restrict__ out, int64_t* __restrict__ count) {
    __shared__ int64_t tmp[kCompBlock / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kComp2Tile + (int64_t)threadIdx.x * kComp2Items;
    int64_t v[kComp2Items];
    typename F::value_type val[kComp2Items];
    int64_t tg[kComp2Items];
    F g = f;
    g.begin(base);
#pragma unroll
    for (int i = 0; i < kComp2Items; i++) {
        v[i] = (base + i < n && g.eval(base + i, val[i])) ? 1 : 0;
        tg[i] = (base + i < n) ? g.tag(base + i) : -1;
    }
    int64_t hit[kComp2Items];
#pragma unroll
    for (int i = 0; i < kComp2Items; i++) hit[i] = v[i];
    int64_t tot = block_exclusive_scan<int64_t, kCompBlock, kComp2Items>(v, tmp);
    int64_t off = offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kComp2Items; i++) {
        if (tg[i] >= 0) g.at(tg[i], off + v[i]);
        if (hit[i]) out[off + v[i]] = val[i];
    }
    if (count && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *count = off + tot;
}

// Runs the two passes; *count_dev receives the kept count (device memory).
// A functor may know, on the device, where its index space really ends (the
// host passes a bound): `__device__ int64_t end() const`.
template <class F, class = void>
struct has_end : std::false_type {};
template <class F>
struct has_end<F, std::void_t<decltype(std::declval<const F&>().end())>> : std::true_type {};

template <class F>
__device__ __forceinline__ int64_t index_end(const F& f, int64_t n) {
    if constexpr (has_end<F>::value) {
        int64_t e = f.end();
        return e < n ? e : n;
    } else {
        return n;
    }
}

// Single-pass ordered compaction with decoupled look-back.  Blocks take
// tiles of kCompTile indices in order from a counter and stop at the index
// space's real end.  Each tile publishes its kept count (flag AGG), finds
// its exclusive offset by summing predecessors back to the first one whose
// inclusive prefix is known (flag PRE), publishes its own prefix, then
// writes.  A tile only waits on tiles taken before it, by blocks that are
// already running, so the wait ends; it is still bounded, and running out
// sets g_lookback_err (never expected), which the caller turns into an error.
constexpr unsigned long long kLbAgg = 1ull << 62, kLbPre = 2ull << 62, kLbVal = (1ull << 62) - 1;
constexpr int kLbSpins = 1 << 24;
static __device__ int g_lookback_err;

// The exclusive prefix of tile t >= 1, by the 32 lanes of one warp: each
// round reads the status words of the 32 tiles before the window's end at
// once, waits (bounded) until each has published, and stops at the nearest
// one whose inclusive prefix is known, summing the aggregates after it.
__device__ __forceinline__ int64_t lookback_prefix_warp(unsigned long long* st, int64_t t) {
    const int lane = threadIdx.x & 31;
    int64_t excl = 0;
    for (int64_t hi = t - 1;; hi -= 32) {
        const int64_t p = hi - lane;
        unsigned long long w = kLbPre;                 // before tile 0: a prefix of 0
        if (p >= 0) {
            int spins = 0;
            for (;;) {
                w = *(volatile unsigned long long*)(st + p);
                if (w >> 62) break;
                if (++spins > kLbSpins) { atomicExch(&g_lookback_err, 1); w = kLbPre; break; }
                __nanosleep(32);
            }
        }
        const unsigned pre = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        const int stop = pre ? __ffs(pre) - 1 : 31;    // the nearest prefix (lane 0 is tile hi)
        int64_t v = lane <= stop ? (int64_t)(w & kLbVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pre) break;
    }
    return excl;
}

// Warp 0 of a block: publish tile t's count `tot` (t relative to its
// index space's first tile, status words st), find its exclusive offset and
// publish its inclusive prefix.  Returns the offset on every lane of warp 0.
__device__ __forceinline__ int64_t tile_publish(unsigned long long* st, int64_t t, int64_t tot) {
    const int lane = threadIdx.x & 31;
    int64_t excl = 0;
    if (t == 0) {
        if (lane == 0) atomicExch(st, kLbPre | (unsigned long long)tot);
    } else {
        if (lane == 0) atomicExch(st + t, kLbAgg | (unsigned long long)tot);
        excl = lookback_prefix_warp(st, t);
        if (lane == 0) atomicExch(st + t, kLbPre | (unsigned long long)(excl + tot));
    }
    return excl;
}

// The last r in [0, rows) with e_off[r] <= i (e_off non-decreasing,
// e_off[0] <= i < e_off[rows]), by the 32 lanes of a warp together: each
// round probes 32 points of the interval at once and keeps the 1/33 between
// two of them, so a search over a million rows takes four rounds of
// parallel loads instead of twenty dependent ones.  Every lane returns it.
__device__ __forceinline__ int64_t warp_row_of(const int64_t* __restrict__ e_off, int64_t rows, int64_t i) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = rows;                            // e_off[lo] <= i < e_off[hi]
    while (hi - lo > 1) {
        const int64_t span = hi - lo;
        const int64_t p = lo + (span * (lane + 1)) / 33;  // non-decreasing in the lane, in [lo, hi)
        const unsigned m = __ballot_sync(0xffffffffu, e_off[p] <= i);
        const int c = __popc(m);                          // the probes with e_off <= i form a prefix
        const int64_t plo = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0);
        const int64_t phi = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
        if (c > 0) lo = plo;                              // e_off[plo] <= i
        if (c < 32) hi = phi;                             // e_off[phi] > i, so phi > plo
    }
    return lo;
}

// The rows of two indices i <= j of the same offsets at once: the two
// 33-way searches of warp_row_of advance together, so each round's probes
// of both are loaded in one go.  A search that has finished keeps probing
// its own row, which leaves it where it is.
__device__ __forceinline__ void warp_rows_of(const int64_t* __restrict__ e_off, int64_t rows, int64_t i, int64_t j,
                                             int64_t* ri, int64_t* rj) {
    const int lane = threadIdx.x & 31;
    int64_t alo = 0, ahi = rows, blo = 0, bhi = rows;
    while (ahi - alo > 1 || bhi - blo > 1) {
        const int64_t pa = alo + ((ahi - alo) * (lane + 1)) / 33;
        const int64_t pb = blo + ((bhi - blo) * (lane + 1)) / 33;
        const int64_t va = e_off[pa], vb = e_off[pb];
        const int ca = __popc(__ballot_sync(0xffffffffu, va <= i));
        const int cb = __popc(__ballot_sync(0xffffffffu, vb <= j));
        const int64_t alo2 = __shfl_sync(0xffffffffu, pa, ca > 0 ? ca - 1 : 0);
        const int64_t ahi2 = __shfl_sync(0xffffffffu, pa, ca < 32 ? ca : 31);
        const int64_t blo2 = __shfl_sync(0xffffffffu, pb, cb > 0 ? cb - 1 : 0);
        const int64_t bhi2 = __shfl_sync(0xffffffffu, pb, cb < 32 ? cb : 31);
        if (ca > 0) alo = alo2;
        if (ca < 32) ahi = ahi2;
        if (cb > 0) blo = blo2;
        if (cb < 32) bhi = bhi2;
    }
    *ri = alo;
    *rj = blo;
}

// A functor may narrow its per-thread setup with a hint computed once per
// tile: `__device__ void tile_hint(int64_t tb, int64_t te, int64_t* h)` (by
// the 32 lanes of warp 0 together; lane 0 writes h[0..1]) and `__device__
// void begin(int64_t i0, const int64_t* h)` (by every thread).  Functors
// without it get begin(i0).
template <class F, class = void>
struct has_hint : std::false_type {};
template <class F>
struct has_hint<F, std::void_t<decltype(std::declval<F&>().tile_hint(int64_t(0), int64_t(0), (int64_t*)nullptr))>>
    : std::true_type {};

template <class F>
__device__ __forceinline__ void tile_hint_of(F& g, int64_t tb, int64_t te, int64_t* h) {
    if constexpr (has_hint<F>::value) g.tile_hint(tb, te, h);
}

template <class F>
__device__ __forceinline__ void begin_with(F& g, int64_t i0, const int64_t* h) {
    if constexpr (has_hint<F>::value) g.begin(i0, h);
    else g.begin(i0);
}

// A functor may also evaluate kEvalN consecutive indices at once, so that
// their independent loads are in flight together:
//   template <int N> __device__ void eval_n(int64_t i0, int64_t end,
//       uint32_t& keep, value_type (&val)[N], int32_t (&tag)[N])
// sets bit j of keep, val[j] and tag[j] (-1: none) as eval(i0 + j) and
// tag(i0 + j) would, for i0 + j < end (bits and tags of the others clear).
template <class F, class = void>
struct has_eval_n : std::false_type {};
template <class F>
struct has_eval_n<F, std::void_t<decltype(std::declval<F&>().template eval_n<kEvalN>(
                         int64_t(0), int64_t(0), std::declval<uint32_t&>(),
                         std::declval<typename F::value_type (&)[kEvalN]>(), std::declval<int32_t (&)[kEvalN]>()))>>
    : std::true_type {};

// Shared memory of a compaction block: the scan's warp totals, the tile's
// description, and each index's value and tag staged between evaluation
// and writing (so that a thread's 16 indices need few registers).
struct CompShared {
    int32_t tmp[kCompBlock / 32 + 1];
    int64_t t, end, first, excl, hint[2];
    int seg;
    uint32_t val[kCompBlock * kCompItems];
    int32_t tag[kCompBlock * kCompItems];
};

// One tile [tb, tb + kCompTile) of an index space ending at `end`: evaluate
// (values and tags staged in shared memory, the kept indices as a bit mask),
// scan the threads' kept counts, publish and look back through the status
// words `st` of the index space (tile lt of it), write.  Every thread of the
// block calls it; `g` has had its begin().
template <class F>
__device__ __forceinline__ void compact_tile(F& g, int64_t tb, int64_t end, unsigned long long* st, int64_t lt,
                                             typename F::value_type* __restrict__ out, int64_t* count,
                                             CompShared& sh) {
    using V = typename F::value_type;
    static_assert(sizeof(V) == 4, "staged values are 32-bit");
    const int64_t base = tb + (int64_t)threadIdx.x * kCompItems;
    V* sv = (V*)(sh.val + threadIdx.x);          // index i of this thread at [i * kCompBlock]:
    int32_t* st_ = sh.tag + threadIdx.x;         // a warp's stores hit 32 distinct banks
    uint32_t hit = 0;
    if constexpr (has_eval_n<F>::value) {
#pragma unroll
        for (int h = 0; h < kCompItems; h += kEvalN) {
            V val[kEvalN];
            int32_t tg[kEvalN];
            uint32_t k = 0;
            g.template eval_n<kEvalN>(base + h, end, k, val, tg);
#pragma unroll
            for (int i = 0; i < kEvalN; i++) { sv[(h + i) * kCompBlock] = val[i]; st_[(h + i) * kCompBlock] = tg[i]; }
            hit |= k << h;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kCompItems; i++) {
            const bool in = base + i < end;
            V x{};
            const bool k = in && g.eval(base + i, x);
            sv[i * kCompBlock] = x;
            hit |= (k ? 1u : 0u) << i;
            st_[i * kCompBlock] = in ? (int32_t)g.tag(base + i) : -1;    // rows and tags are below 2^31
        }
    }
    int32_t mine[1] = {__popc(hit)};
    const int32_t tot = block_exclusive_scan<int32_t, kCompBlock, 1>(mine, sh.tmp);
    if (threadIdx.x < 32) {
        const int64_t excl = tile_publish(st, lt, (int64_t)tot);
        if (threadIdx.x == 0) {
            sh.excl = excl;
            if (tb + kCompTile >= end && count) *count = excl + tot;   // the last tile
        }
    }
    __syncthreads();
    const int64_t off = sh.excl + mine[0];
    int32_t r = 0;
#pragma unroll
    for (int i = 0; i < kCompItems; i++) {
        const int32_t t = st_[i * kCompBlock];
        if (t >= 0) g.at((int64_t)t, off + r);
        if ((hit >> i) & 1u) out[off + r++] = sv[i * kCompBlock];
    }
    __syncthreads();
}

template <class F>
__global__ void __launch_bounds__(kCompBlock, kCompBlocksPerSM) k_compact_1p(F f, int64_t n, typename F::value_type* __restrict__ out,
                                                              int64_t* __restrict__ count,
                                                              unsigned long long* __restrict__ st,
                                                              unsigned int* __restrict__ tile_ctr) {
    __shared__ CompShared sh;
    if (threadIdx.x == 0) sh.end = index_end(f, n);
    __syncthreads();
    const int64_t end = sh.end;
    for (;;) {
        if (threadIdx.x < 32) {                           // warp 0: take a tile, find its hint
            int64_t t = 0;
            if (threadIdx.x == 0) t = (int64_t)atomicAdd(tile_ctr, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            const int64_t tb = t * kCompTile;
            if (tb < end) tile_hint_of(f, tb, tb + kCompTile < end ? tb + kCompTile : end, sh.hint);
            if (threadIdx.x == 0) sh.t = t;
        }
        __syncthreads();
        const int64_t t = sh.t;
        const int64_t tb = t * kCompTile;
        if (tb >= end) {
            if (t == 0 && threadIdx.x == 0 && count) *count = 0;     // empty index space
            break;
        }
        F g = f;
        begin_with(g, tb + (int64_t)threadIdx.x * kCompItems, sh.hint);
        compact_tile(g, tb, end, st, t, out, count, sh);
    }
}

template <class F>
int compact(const F& f, int64_t n, typename F::value_type* out, int64_t* count_dev, cudaStream_t s) {
    if (n <= 0) {
        if (count_dev) FAST_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int64_t), s));
        return FAST_OK;
    }
    const int64_t nt = ceil_div(n, kCompTile);
    unsigned long long* st = nullptr;                     // [nt] tile status, then the tile counter
    FAST_TRY(dalloc(&st, nt + 1, s));
    cudaMemsetAsync(st, 0, (nt + 1) * sizeof(unsigned long long), s);
    const int64_t grid = std::min<int64_t>(nt, (int64_t)num_sms() * kCompBlocksPerSM);
    k_compact_1p<F><<<(unsigned)grid, kCompBlock, 0, s>>>(f, n, out, count_dev, st, (unsigned int*)(st + nt));
    note_launch();
    int rc = cudaGetLastError() == cudaSuccess ? FAST_OK : set_error(FAST_ERR_CUDA, "compaction launch");
    dfree(st, s);
    return rc;
}


template <class F>
int compact_alloc(const F& f, int64_t n, typename F::value_type** out, int64_t* kept_host, cudaStream_t s) {
    *out = nullptr;
    *kept_host = 0;
    if (n <= 0) return FAST_OK;
    int64_t nb = ceil_div(n, kComp2Tile);
    int64_t* offs = nullptr;
    int64_t* tot = nullptr;
    FAST_TRY(dalloc(&offs, nb + 1, s));
    tot = offs + nb;
    int rc = FAST_OK;
    k_compact_count<F><<<(unsigned)nb, kCompBlock, 0, s>>>(f, n, offs);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "compact count launch");
    if (rc == FAST_OK) rc = scan_exclusive<int64_t>(offs, offs, nb, tot, s);
    if (rc == FAST_OK) {
        cudaError_t e = cudaMemcpyAsync(kept_host, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e, "compaction size readback", __FILE__, __LINE__);
    }
    if (rc == FAST_OK) rc = dalloc(out, (size_t)(*kept_host), s);
    if (rc == FAST_OK) {
        k_compact_write<F><<<(unsigned)nb, kCompBlock, 0, s>>>(f, n, offs, *out, (int64_t*)nullptr);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "compact write launch");
    }
    dfree(offs, s);
    if (rc != FAST_OK) dfree(*out, s);
    return rc;
}

// --------------------------------------------------------------- radix sort
//
// Stable LSD radix sort of uint64 keys, 8-bit digits, over the digit
// positions listed in `shifts`.  Three kernels per pass: per-tile digit
// histograms, a digit-major exclusive scan of them, and a stable scatter that
// ranks keys inside a tile warp by warp with __match_any_sync.

constexpr int kSortBlock = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortBlock * kSortRounds;

static __global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t nblocks,
                             uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = base + (int64_t)r * kSortBlock + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

static __global__ void k_radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n,
                                int shift, int64_t nblocks, const uint32_t* __restrict__ offs) {
    constexpr int NW = kSortBlock / 32;
    __shared__ uint32_t goff[256];        // global start of this tile's digit run
    __shared__ uint32_t run[256];         // keys of each digit already placed
    __shared__ uint32_t wcnt[NW][256];    // per-round per-warp counts -> offsets
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    goff[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    run[threadIdx.x] = 0;
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; r++) {
#pragma unroll
        for (int w = 0; w < NW; w++) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * kSortBlock + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? in[i] : 0;
        uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : 256u + lane;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t b = run[threadIdx.x];
#pragma unroll
            for (int w = 0; w < NW; w++) {
                uint32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = b;
                b += c;
            }
            run[threadIdx.x] = b;
        }
        __syncthreads();
        if (valid) out[goff[d] + wcnt[warp][d] + rank] = key;
        __syncthreads();
    }
}

// Sorts keys[0..n) in place (tmp: caller scratch of n keys, or null to
// allocate).  n must be below 2^32.
inline int radix_sort_u64(uint64_t* keys, int64_t n, const int* shifts, int npass, cudaStream_t s) {
    if (n <= 1 || npass == 0) return FAST_OK;
    if (n >= (int64_t)0xFFFFFFFFll) return set_error(FAST_ERR_INVALID, "radix sort: too many keys (%lld)", (long long)n);
    int64_t nb = ceil_div(n, kSortTile);
    uint64_t* tmp = nullptr;
    uint32_t* hist = nullptr;
    FAST_TRY(dalloc(&tmp, n, s));
    int rc = dalloc(&hist, 256 * nb, s);
    uint64_t* a = keys;
    uint64_t* b = tmp;
    for (int p = 0; p < npass && rc == FAST_OK; p++) {
        k_radix_hist<<<(unsigned)nb, kSortBlock, 0, s>>>(a, n, shifts[p], nb, hist);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "radix hist launch"); break; }
        rc = scan_exclusive<uint32_t>(hist, hist, 256 * nb, (uint32_t*)nullptr, s);
        if (rc != FAST_OK) break;
        k_radix_scatter<<<(unsigned)nb, kSortBlock, 0, s>>>(a, b, n, shifts[p], nb, hist);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) { rc = set_error(FAST_ERR_CUDA, "radix scatter launch"); break; }
        uint64_t* t = a; a = b; b = t;
    }
    if (rc == FAST_OK && a != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, a, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) rc = cuda_status(e, "radix copy back", __FILE__, __LINE__);
    }
    dfree(tmp, s);
    dfree(hist, s);
    return rc;
}

// Digit shifts covering bits [lo, hi) in 8-bit steps.
inline int digit_shifts(int lo, int hi, int* out, int max_out) {
    int n = 0;
    for (int sft = lo; sft < hi && n < max_out; sft += 8) out[n++] = sft;
    return n;
}

inline int bits_for(int64_t maxval) {
    int b = 0;
    while (b < 63 && (maxval >> b) > 0) b++;
    return b;
}

}  // namespace fast
