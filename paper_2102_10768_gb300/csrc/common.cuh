// Internal helpers shared by the library's translation units: status
// handling, the last-error message, stream-ordered allocation and small
// device utilities.  Nothing here is part of the C ABI (see include/fast.h).
#pragma once

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

#define FAST_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess) return ::fast::cuda_status(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define FAST_TRY(call)                    \
    do {                                  \
        int _rc = (call);                 \
        if (_rc != FAST_OK) return _rc;   \
    } while (0)

// Stream-ordered device allocation; n == 0 yields a valid 256-byte block so
// that kernels may always receive a non-null pointer.
template <class T>
inline int dalloc(T** p, size_t n, cudaStream_t s) {
    size_t bytes = n * sizeof(T);
    if (bytes == 0) bytes = 256;
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
inline void dfree(T*& p, cudaStream_t s) {
    if (p) cudaFreeAsync((void*)p, s);
    p = nullptr;
}

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
