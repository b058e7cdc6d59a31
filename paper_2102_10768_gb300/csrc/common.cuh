// Internal helpers shared by the library's translation units: status
// handling, the last-error message, device memory (stream-ordered
// allocation, scratch pools, arenas) and small device utilities.  Nothing here is part of the C ABI (see include/fast.h).
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/fast.h"

namespace fast {

// Records a message for fast_last_error() (thread local) and returns code.
int set_error(int code, const char* fmt, ...);

// Counts kernel launches made by the library (fast_kernel_launches()).
void note_launch(int n = 1);

// Turns a CUDA error into FAST_ERR_OOM / FAST_ERR_CUDA with a message.
int cuda_status(cudaError_t e, const char* what, const char* file, int line);

// Allocation-failure injection (fast_inject_alloc_failure): true for the
// one device allocation the armed countdown reaches, which then fails with
// FAST_ERR_OOM.  Disarmed, it costs one relaxed atomic load.
bool alloc_fault_due();

#define FAST_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess) return ::fast::cuda_status(_e, #call, __FILE__, __LINE__); \
    } while (0)

// For a `do { ... } while (0)` block with cleanup after it: on a CUDA error,
// stores the status in rc and leaves the block instead of returning.
#define FAST_CUDA_BREAK(rc, call)                                                          \
    {                                                                                      \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) { (rc) = ::fast::cuda_status(_e, #call, __FILE__, __LINE__); break; } \
    }

#define FAST_TRY(call)                    \
    do {                                  \
        int _rc = (call);                 \
        if (_rc != FAST_OK) return _rc;   \
    } while (0)

// ------------------------------------------------------- device memory
//
// dalloc/dfree: temporaries.  Inside a PoolScope they come from the bound
// ScratchPool (pool.cu); elsewhere from the stream-ordered allocator.
// dalloc_direct/dfree_direct: memory that outlives the call (always the
// stream-ordered allocator).  Arena: a CST's own arrays, bump-allocated from
// a few large blocks and returned together.
struct ScratchPool;
ScratchPool* pool_new();
void pool_delete(ScratchPool* p);
void retain_freed_memory();                                  // once per device: keep freed memory pooled
void pool_release_unused(ScratchPool* p);                    // free the scratch blocks with no live region
void trim_freed_memory();                                    // give the pooled memory back
ScratchPool* pool_active();                                  // bound to this thread, or null
int pool_alloc(ScratchPool* p, void** out, size_t bytes);
bool pool_free(ScratchPool* p, void* ptr);                   // false: not from this pool

// Binds a pool to this thread for a scope: `p`, else the one already bound,
// else this thread's default pool for the current device.  On exit, if the
// pool handed out memory meanwhile, synchronises `s`: a region freed in the
// scope may still be read by work queued on `s`, and must be idle before the
// pool serves any other call.
class PoolScope {
  public:
    explicit PoolScope(cudaStream_t s, ScratchPool* p = nullptr);
    ~PoolScope();
    PoolScope(const PoolScope&) = delete;
    PoolScope& operator=(const PoolScope&) = delete;

  private:
    ScratchPool* prev_;
    ScratchPool* cur_;
    cudaStream_t s_;
    uint64_t mark_;
};

// n == 0 yields a valid 256-byte block so that kernels may always receive a
// non-null pointer.
template <class T>
inline int dalloc_direct(T** p, size_t n, cudaStream_t s) {
    size_t bytes = n * sizeof(T);
    if (bytes == 0) bytes = 256;
    if (alloc_fault_due()) {
        *p = nullptr;
        return set_error(FAST_ERR_OOM, "device allocation of %zu bytes failed: injected", bytes);
    }
    retain_freed_memory();
    cudaError_t e = cudaMallocAsync((void**)p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(FAST_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    return FAST_OK;
}

template <class T>
inline void dfree_direct(T*& p, cudaStream_t s) {
    if (p) cudaFreeAsync((void*)p, s);
    p = nullptr;
}

template <class T>
inline int dalloc(T** p, size_t n, cudaStream_t s) {
    if (ScratchPool* sp = pool_active()) {
        size_t bytes = n * sizeof(T);
        return pool_alloc(sp, (void**)p, bytes ? bytes : 256);
    }
    return dalloc_direct(p, n, s);
}

template <class T>
inline void dfree(T*& p, cudaStream_t s) {
    if (p) {
        ScratchPool* sp = pool_active();
        if (!sp || !pool_free(sp, (void*)p)) cudaFreeAsync((void*)p, s);
    }
    p = nullptr;
}

class Arena {
  public:
    template <class T>
    int alloc(T** p, size_t n, cudaStream_t s) {
        size_t bytes = n * sizeof(T);
        bytes = bytes ? (bytes + 255) / 256 * 256 : 256;
        if (bytes > left_) {
            int rc = grow(bytes, s);
            if (rc != FAST_OK) { *p = nullptr; return rc; }
        }
        *p = (T*)cur_;
        cur_ += bytes;
        left_ -= bytes;
        return FAST_OK;
    }
    // one block of exactly `bytes` (256-byte multiple) when the arena is empty
    template <class T>
    int alloc_exact(T** p, size_t bytes, cudaStream_t s) {
        if (blocks_.empty() && bytes > 0) next_ = (bytes + 255) / 256 * 256;
        *p = nullptr;
        return alloc((unsigned char**)p, bytes, s);
    }
    void release(cudaStream_t s);

  private:
    int grow(size_t bytes, cudaStream_t s);
    std::vector<void*> blocks_;
    char* cur_ = nullptr;
    size_t left_ = 0;
    size_t next_ = 16ull << 20;
};

inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------ device side

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__host__ __device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return s < a ? ~0ull : s;
}

__host__ __device__ __forceinline__ uint64_t sat_mul(uint64_t a, uint64_t b) {
    if (a == 0 || b == 0) return 0;
#ifdef __CUDA_ARCH__
    uint64_t hi = __umul64hi(a, b);
    return hi ? ~0ull : a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    return (p >> 64) ? ~0ull : (uint64_t)p;
#endif
}

// splitmix64 finaliser (Steele, Lea, Flood 2014); used for the seeded
// sampling of partitions, identically on host and device.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace fast
