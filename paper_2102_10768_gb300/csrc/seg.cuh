// Segmented twins of the single-pass ordered compaction and exclusive scan
// (prims.cuh): many independent index spaces ("segments": one per query of a
// batch, or per query edge) in one launch.
//
// The tiles of all segments form one global tile sequence: segment s owns
// tiles tile_off[s] .. tile_off[s+1]-1 (at least one, so that an empty
// segment still reports a zero count).  Blocks of a persistent grid take
// tiles in that order from one counter.  A tile publishes its aggregate and
// looks back over the earlier tiles of its own segment only, stopping at the
// segment's first tile; every tile it waits on was taken before it by a
// block that is already running, so the wait ends.  It is still bounded by
// the same spin limit as the single-segment form, and running out sets the
// translation unit's look-back error flag.
#pragma once

#include <vector>

#include "prims.cuh"

namespace fast {

// last s with tile_off[s] <= t (the segment owning tile t; the empty
// segments before it share its offset)
__device__ __forceinline__ int seg_of_tile(const int64_t* __restrict__ tile_off, int nseg, int64_t t) {
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Host side: tile_off[0..nseg] for segments of n_s indices, tiles of `tile`
// indices, at least one tile per segment.
inline std::vector<int64_t> seg_tile_offsets(const std::vector<int64_t>& n, int64_t tile) {
    std::vector<int64_t> off(n.size() + 1, 0);
    for (size_t i = 0; i < n.size(); i++) off[i + 1] = off[i] + std::max<int64_t>(1, ceil_div(n[i], tile));
    return off;
}

// One scratch block holding, in order: the descriptors, the tile offsets,
// the tile status words and the tile counter.  Uploads the first two with
// one copy and zeroes the rest with one memset.
struct SegBlock {
    unsigned char* base = nullptr;
    size_t desc_bytes = 0, off_at = 0, st_at = 0, bytes = 0;
    int64_t tiles = 0;
};

template <class D>
int seg_block_upload(const std::vector<D>& desc, const std::vector<int64_t>& tile_off, SegBlock* b, cudaStream_t s) {
    const size_t nd = desc.size();
    b->tiles = tile_off.back();
    b->desc_bytes = nd * sizeof(D);
    b->off_at = (b->desc_bytes + 15) / 16 * 16;
    b->st_at = (b->off_at + tile_off.size() * sizeof(int64_t) + 15) / 16 * 16;
    b->bytes = b->st_at + (size_t)(b->tiles + 1) * sizeof(unsigned long long);
    FAST_TRY(dalloc(&b->base, b->bytes, s));
    std::vector<unsigned char> h(b->st_at, 0);
    memcpy(h.data(), desc.data(), b->desc_bytes);
    memcpy(h.data() + b->off_at, tile_off.data(), tile_off.size() * sizeof(int64_t));
    FAST_CUDA(cudaMemcpyAsync(b->base, h.data(), b->st_at, cudaMemcpyHostToDevice, s));
    FAST_CUDA(cudaMemsetAsync(b->base + b->st_at, 0, b->bytes - b->st_at, s));
    return FAST_OK;
}

// ------------------------------------------------------------- compaction

template <class F>
struct CompactSeg {
    F f;
    int64_t n;                                // index space [0, n) (a bound when F has end())
    typename F::value_type* out;
    int64_t* count;                           // device, nullable: kept indices
};

template <class F>
__global__ void __launch_bounds__(kCompBlock, kCompBlocksPerSM) k_compact_seg(const CompactSeg<F>* __restrict__ segs,
                                                               const int64_t* __restrict__ tile_off, int nseg,
                                                               unsigned long long* __restrict__ st,
                                                               unsigned int* __restrict__ tile_ctr) {
    __shared__ CompShared sh;
    const int64_t total = tile_off[nseg];
    for (;;) {
        if (threadIdx.x < 32) {                           // warp 0: take a tile, find its segment and hint
            int64_t t = 0, first = 0, end = 0;
            int sg = 0;
            if (threadIdx.x == 0) {
                t = (int64_t)atomicAdd(tile_ctr, 1u);
                if (t < total) {
                    sg = seg_of_tile(tile_off, nseg, t);
                    first = tile_off[sg];
                    end = index_end(segs[sg].f, segs[sg].n);
                }
            }
            t = __shfl_sync(0xffffffffu, t, 0);
            sg = __shfl_sync(0xffffffffu, sg, 0);
            first = __shfl_sync(0xffffffffu, first, 0);
            end = __shfl_sync(0xffffffffu, end, 0);
            const int64_t tb = (t - first) * kCompTile;
            if (t < total && tb < end) {
                F h = segs[sg].f;
                tile_hint_of(h, tb, tb + kCompTile < end ? tb + kCompTile : end, sh.hint);
            }
            if (threadIdx.x == 0) { sh.t = t; sh.seg = sg; sh.first = first; sh.end = end; }
        }
        __syncthreads();
        const int64_t t = sh.t;
        if (t >= total) break;
        const CompactSeg<F>& sd = segs[sh.seg];
        const int64_t lt = t - sh.first, end = sh.end;
        const int64_t tb = lt * kCompTile;
        if (tb >= end) {                                   // past the segment's real end
            if (lt == 0 && threadIdx.x == 0 && sd.count) *sd.count = 0;
            __syncthreads();
            continue;
        }
        F g = sd.f;
        begin_with(g, tb + (int64_t)threadIdx.x * kCompItems, sh.hint);
        compact_tile(g, tb, end, st + sh.first, lt, sd.out, sd.count, sh);
    }
}

// All segments in one launch; each segment's kept count goes to its
// `count` (device).
template <class F>
int compact_seg(const std::vector<CompactSeg<F>>& segs, cudaStream_t s) {
    if (segs.empty()) return FAST_OK;
    std::vector<int64_t> n(segs.size());
    for (size_t i = 0; i < segs.size(); i++) n[i] = segs[i].n;
    const std::vector<int64_t> toff = seg_tile_offsets(n, kCompTile);
    SegBlock b;
    int rc = seg_block_upload(segs, toff, &b, s);
    if (rc == FAST_OK) {
        const int64_t grid = std::min<int64_t>(b.tiles, (int64_t)num_sms() * kCompBlocksPerSM);
        k_compact_seg<F><<<(unsigned)grid, kCompBlock, 0, s>>>(
            (const CompactSeg<F>*)b.base, (const int64_t*)(b.base + b.off_at), (int)segs.size(),
            (unsigned long long*)(b.base + b.st_at), (unsigned int*)(b.base + b.st_at + b.tiles * sizeof(unsigned long long)));
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "segmented compaction launch");
    }
    dfree(b.base, s);
    return rc;
}

// ------------------------------------------------------- bitmap -> ids
//
// The ids of the set bits of each segment's bitmap (bits [0, nbits)), in
// increasing order, and their number: a compaction over 32-bit words, whose
// tiles count their words' bits, find their offsets by the same look-back,
// then write each word's ids.

struct BitsSeg {
    const uint32_t* bits;
    int64_t nbits;
    int32_t* out;
    int64_t* count;                           // device, nullable
};

constexpr int kBitsItems = 8;                 // words per thread
constexpr int kBitsTile = kCompBlock * kBitsItems;

static __global__ void __launch_bounds__(kCompBlock, kCompBlocksPerSM) k_bits_ids_seg(const BitsSeg* __restrict__ segs,
                                                             const int64_t* __restrict__ tile_off, int nseg,
                                                             unsigned long long* __restrict__ st,
                                                             unsigned int* __restrict__ tile_ctr) {
    __shared__ int64_t tmp[kCompBlock / 32 + 1];
    __shared__ int64_t s_t, s_excl, s_first;
    __shared__ int s_seg;
    const int64_t total = tile_off[nseg];
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(tile_ctr, 1u);
            s_t = t;
            if (t < total) {
                const int sg = seg_of_tile(tile_off, nseg, t);
                s_seg = sg;
                s_first = tile_off[sg];
            }
        }
        __syncthreads();
        const int64_t t = s_t;
        if (t >= total) break;
        const BitsSeg& sd = segs[s_seg];
        const int64_t lt = t - s_first;
        const int64_t nw = (sd.nbits + 31) >> 5;
        const int64_t tb = lt * kBitsTile;
        if (tb >= nw) {                                   // an empty bitmap
            if (lt == 0 && threadIdx.x == 0 && sd.count) *sd.count = 0;
            __syncthreads();
            continue;
        }
        const int64_t base = tb + (int64_t)threadIdx.x * kBitsItems;
        uint32_t w[kBitsItems];
        int64_t v[kBitsItems];
#pragma unroll
        for (int i = 0; i < kBitsItems; i++) {
            const int64_t x = base + i;
            uint32_t b = x < nw ? sd.bits[x] : 0u;
            if (x == nw - 1 && (sd.nbits & 31)) b &= (1u << (sd.nbits & 31)) - 1u;   // bits past nbits
            w[i] = b;
            v[i] = __popc(b);
        }
        const int64_t tot = block_exclusive_scan<int64_t, kCompBlock, kBitsItems>(v, tmp);
        if (threadIdx.x < 32) {
            const int64_t excl = tile_publish(st + s_first, lt, tot);
            if (threadIdx.x == 0) {
                s_excl = excl;
                if (tb + kBitsTile >= nw && sd.count) *sd.count = excl + tot;
            }
        }
        __syncthreads();
        int64_t o = s_excl + v[0];
        int32_t* out = sd.out;
#pragma unroll
        for (int i = 0; i < kBitsItems; i++) {
            uint32_t b = w[i];
            const int32_t id0 = (int32_t)((base + i) << 5);
            while (b) {
                out[o++] = id0 + (__ffs(b) - 1);
                b &= b - 1;
            }
        }
        __syncthreads();
    }
}

inline int bits_ids_seg(const std::vector<BitsSeg>& segs, cudaStream_t s) {
    if (segs.empty()) return FAST_OK;
    std::vector<int64_t> nw(segs.size());
    for (size_t i = 0; i < segs.size(); i++) nw[i] = (segs[i].nbits + 31) >> 5;
    const std::vector<int64_t> toff = seg_tile_offsets(nw, kBitsTile);
    SegBlock b;
    int rc = seg_block_upload(segs, toff, &b, s);
    if (rc == FAST_OK) {
        const int64_t grid = std::min<int64_t>(b.tiles, (int64_t)num_sms() * kCompBlocksPerSM);
        k_bits_ids_seg<<<(unsigned)grid, kCompBlock, 0, s>>>(
            (const BitsSeg*)b.base, (const int64_t*)(b.base + b.off_at), (int)segs.size(),
            (unsigned long long*)(b.base + b.st_at), (unsigned int*)(b.base + b.st_at + b.tiles * sizeof(unsigned long long)));
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "bitmap ids launch");
    }
    dfree(b.base, s);
    return rc;
}

// ------------------------------------------------------------------- scan

// out[i] = in[0] + ... + in[i-1] over [0, n); *total (nullable) = the sum.
// With `bits` set, in[i] = popcount(bits[i]) (the rank of a bitmap's words).
// in and out may alias.
template <class T>
struct ScanSeg {
    const T* in;
    const uint32_t* bits;
    T* out;
    int64_t n;
    T* total;
};

template <class T>
__global__ void __launch_bounds__(kScanBlock) k_scan_seg(const ScanSeg<T>* __restrict__ segs,
                                                         const int64_t* __restrict__ tile_off, int nseg,
                                                         unsigned long long* __restrict__ st,
                                                         unsigned int* __restrict__ tile_ctr) {
    __shared__ T tmp[kScanBlock / 32 + 1];
    __shared__ int64_t s_t, s_excl, s_first;
    __shared__ int s_seg;
    const int64_t total = tile_off[nseg];
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(tile_ctr, 1u);
            s_t = t;
            if (t < total) {
                const int sg = seg_of_tile(tile_off, nseg, t);
                s_seg = sg;
                s_first = tile_off[sg];
            }
        }
        __syncthreads();
        const int64_t t = s_t;
        if (t >= total) break;
        const ScanSeg<T>& sd = segs[s_seg];
        const int64_t lt = t - s_first, n = sd.n;
        const int64_t tb = lt * kScanTile;
        if (tb >= n) {                                     // empty segment
            if (lt == 0 && threadIdx.x == 0 && sd.total) *sd.total = T(0);
            __syncthreads();
            continue;
        }
        const int64_t base = tb + (int64_t)threadIdx.x * kScanItems;
        T v[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; i++) {
            const int64_t x = base + i;
            v[i] = x < n ? (sd.bits ? (T)__popc(sd.bits[x]) : sd.in[x]) : T(0);
        }
        const T tot = block_exclusive_scan<T, kScanBlock, kScanItems>(v, tmp);
        if (threadIdx.x < 32) {
            const int64_t excl = tile_publish(st + s_first, lt, (int64_t)tot);
            if (threadIdx.x == 0) {
                s_excl = excl;
                if (tb + kScanTile >= n && sd.total) *sd.total = (T)(excl + (int64_t)tot);
            }
        }
        __syncthreads();
        const T off = (T)s_excl;
        T* out = sd.out;
#pragma unroll
        for (int i = 0; i < kScanItems; i++)
            if (base + i < n) out[base + i] = v[i] + off;
        __syncthreads();
    }
}

template <class T>
int scan_seg(const std::vector<ScanSeg<T>>& segs, cudaStream_t s) {
    if (segs.empty()) return FAST_OK;
    std::vector<int64_t> n(segs.size());
    for (size_t i = 0; i < segs.size(); i++) n[i] = segs[i].n;
    const std::vector<int64_t> toff = seg_tile_offsets(n, kScanTile);
    SegBlock b;
    int rc = seg_block_upload(segs, toff, &b, s);
    if (rc == FAST_OK) {
        const int64_t grid = std::min<int64_t>(b.tiles, (int64_t)num_sms() * 2);
        k_scan_seg<T><<<(unsigned)grid, kScanBlock, 0, s>>>(
            (const ScanSeg<T>*)b.base, (const int64_t*)(b.base + b.off_at), (int)segs.size(),
            (unsigned long long*)(b.base + b.st_at), (unsigned int*)(b.base + b.st_at + b.tiles * sizeof(unsigned long long)));
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = set_error(FAST_ERR_CUDA, "segmented scan launch");
    }
    dfree(b.base, s);
    return rc;
}

}  // namespace fast
