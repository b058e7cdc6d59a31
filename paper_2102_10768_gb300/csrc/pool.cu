// Device scratch memory for the per-query steps.
//
// A CST build, a partition and a matcher call each allocate and free dozens
// of temporaries (compaction state, bitmaps, bounded list buffers).  Through
// the stream-ordered allocator every pair costs tens of microseconds of host
// time, and host threads building CSTs concurrently contend for it.  A
// ScratchPool keeps a few large device blocks and hands out regions from a
// first-fit free list with coalescing, in host bookkeeping only.
//
// Safety: a region freed during an API call may still be read by kernels
// queued on that call's stream; it is handed out again only to the same call
// (same stream, so the kernels are ordered), and PoolScope synchronises the
// stream before the pool can serve any other call.
#include <atomic>
#include <map>
#include <memory>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fast {

struct ScratchPool {
    struct Block {
        char* base = nullptr;
        size_t size = 0;
        std::map<size_t, size_t> free_;      // offset -> bytes
    };
    int device = -1;
    std::vector<Block> blocks;
    std::unordered_map<char*, std::pair<int, size_t>> live;
    uint64_t served = 0;
};

namespace {

constexpr size_t kPoolAlign = 256;
constexpr size_t kPoolBlock = 256ull << 20;

thread_local ScratchPool* tl_active = nullptr;

struct PoolDeleter {
    void operator()(ScratchPool* p) const { pool_delete(p); }
};
thread_local std::map<int, std::unique_ptr<ScratchPool, PoolDeleter>> tl_default;

ScratchPool* default_pool() {
    int dev = 0;
    cudaGetDevice(&dev);
    auto& slot = tl_default[dev];
    if (!slot) {
        slot.reset(pool_new());
        slot->device = dev;
    }
    return slot.get();
}

}  // namespace

// The stream-ordered allocator's default pool returns freed memory to the
// device at every synchronisation unless told to keep it.  A batched step
// allocates and frees tens of GB of CSTs, so that round trip through the
// driver's page tables would come back every step: keep freed memory in the
// pool, once per device (a setting of this process only).
void retain_freed_memory() {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
    if (dev < 0 || dev >= 64) return;
    const uint64_t bit = 1ull << dev;
    if (done.load(std::memory_order_relaxed) & bit) return;
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.fetch_or(bit, std::memory_order_relaxed);
}

// Give the pool's unused memory back to the device (after a large workload
// ends, e.g. when its graph is freed).
void trim_freed_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, dev) == cudaSuccess) cudaMemPoolTrimTo(mp, 0);
    cudaGetLastError();
}

ScratchPool* pool_new() {
    ScratchPool* p = new ScratchPool();
    cudaGetDevice(&p->device);
    return p;
}

void pool_delete(ScratchPool* p) {
    if (!p) return;
    for (auto& b : p->blocks) cudaFree(b.base);
    delete p;
}

ScratchPool* pool_active() { return tl_active; }

// Free the blocks of p that hold no live region (their memory back to the
// device), e.g. after a build that ran out of memory left them large.
void pool_release_unused(ScratchPool* p) {
    if (!p) return;
    std::vector<ScratchPool::Block> keep;
    for (auto& b : p->blocks) {
        const bool empty = b.free_.size() == 1 && b.free_.begin()->first == 0 && b.free_.begin()->second == b.size;
        if (empty) cudaFree(b.base);
        else keep.push_back(std::move(b));
    }
    // live regions record their block's index: renumber
    for (auto& kv : p->live) {
        for (int i = 0; i < (int)keep.size(); i++)
            if (kv.first >= keep[i].base && kv.first < keep[i].base + keep[i].size) { kv.second.first = i; break; }
    }
    p->blocks = std::move(keep);
}

// Allocations left before the injected failure; negative: disarmed.
std::atomic<int64_t> g_alloc_countdown{-1};

bool alloc_fault_due() {
    if (g_alloc_countdown.load(std::memory_order_relaxed) < 0) return false;
    if (g_alloc_countdown.fetch_sub(1, std::memory_order_relaxed) != 0) return false;
    g_alloc_countdown.store(-1, std::memory_order_relaxed);    // one failure, then disarmed
    return true;
}

int pool_alloc(ScratchPool* p, void** out, size_t bytes) {
    if (alloc_fault_due()) {
        *out = nullptr;
        return set_error(FAST_ERR_OOM, "scratch region of %zu bytes: injected failure", bytes);
    }
    bytes = (bytes + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
    for (int pass = 0; pass < 2; pass++) {
        for (int b = 0; b < (int)p->blocks.size(); b++) {
            auto& F = p->blocks[b].free_;
            for (auto it = F.begin(); it != F.end(); ++it) {
                if (it->second < bytes) continue;
                size_t off = it->first, sz = it->second;
                F.erase(it);
                if (sz > bytes) F.emplace(off + bytes, sz - bytes);
                char* ptr = p->blocks[b].base + off;
                p->live.emplace(ptr, std::make_pair(b, bytes));
                p->served++;
                *out = ptr;
                return FAST_OK;
            }
        }
        if (pass == 1) break;
        ScratchPool::Block nb;
        nb.size = bytes > kPoolBlock ? bytes : kPoolBlock;
        cudaError_t e = cudaMalloc((void**)&nb.base, nb.size);
        if (e == cudaErrorMemoryAllocation) {
            // the stream-ordered pool may be holding freed memory: hand it back, try once more
            cudaGetLastError();
            trim_freed_memory();
            e = cudaMalloc((void**)&nb.base, nb.size);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            *out = nullptr;
            return set_error(FAST_ERR_OOM, "scratch block of %zu bytes: %s", nb.size, cudaGetErrorString(e));
        }
        nb.free_.emplace(0, nb.size);
        p->blocks.push_back(std::move(nb));
    }
    *out = nullptr;
    return set_error(FAST_ERR_OOM, "scratch pool: no region of %zu bytes", bytes);
}

bool pool_free(ScratchPool* p, void* ptr) {
    auto it = p->live.find((char*)ptr);
    if (it == p->live.end()) return false;
    int b = it->second.first;
    size_t off = (size_t)((char*)ptr - p->blocks[b].base), sz = it->second.second;
    p->live.erase(it);
    auto& F = p->blocks[b].free_;
    auto nx = F.lower_bound(off);
    if (nx != F.end() && off + sz == nx->first) {
        sz += nx->second;
        nx = F.erase(nx);
    }
    if (nx != F.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            pv->second += sz;
            return true;
        }
    }
    F.emplace(off, sz);
    return true;
}

PoolScope::PoolScope(cudaStream_t s, ScratchPool* p) : s_(s) {
    prev_ = tl_active;
    cur_ = p ? p : (tl_active ? tl_active : default_pool());
    tl_active = cur_;
    mark_ = cur_->served;
}

PoolScope::~PoolScope() {
    if (cur_->served != mark_) cudaStreamSynchronize(s_);
    tl_active = prev_;
}

int Arena::grow(size_t bytes, cudaStream_t s) {
    if (alloc_fault_due()) return set_error(FAST_ERR_OOM, "CST block of %zu bytes: injected failure", bytes);
    size_t sz = bytes;
    if (sz < next_) sz = next_;
    void* b = nullptr;
    retain_freed_memory();
    cudaError_t e = cudaMallocAsync(&b, sz, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(FAST_ERR_OOM, "CST block of %zu bytes: %s", sz, cudaGetErrorString(e));
    }
    blocks_.push_back(b);
    cur_ = (char*)b;
    left_ = sz;
    next_ = sz * 2;
    return FAST_OK;
}

void Arena::release(cudaStream_t s) {
    for (void* b : blocks_) cudaFreeAsync(b, s);
    blocks_.clear();
    cur_ = nullptr;
    left_ = 0;
}

}  // namespace fast

extern "C" int64_t fast_inject_alloc_failure(int64_t after) {
    return fast::g_alloc_countdown.exchange(after < 0 ? -1 : after, std::memory_order_relaxed);
}
