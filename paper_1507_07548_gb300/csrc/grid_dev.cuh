// Bounded grid-wide barrier of the persistent cooperative kernels (k_step.cu,
// batch.cu): a monotone counter per launch, release/acquire at gpu scope, every
// wait limited by %globaltimer.
#pragma once
#include "ms2_internal.cuh"

namespace grid_dev {

constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The k-th barrier of a launch waits for count >= k * gridDim.x.  Ordering: the
// block's writes happen before thread 0's arrival (bar.sync), which is a
// gpu-scope release; thread 0's polling load is a gpu-scope acquire, and the
// closing bar.sync orders the block's later reads after it (release/acquire are
// cumulative in the PTX memory model).  A block that waits longer than wait_ns
// (WAIT_NS unless a test shortens it) sets the sticky flag *err, which ends
// every other wait at once, and calls on_timeout() (thread 0); the kernel then
// runs on without waiting.
template <class OnTimeout>
__device__ __forceinline__ void grid_sync(unsigned *count, unsigned *err, unsigned &target, OnTimeout on_timeout,
                                          unsigned long long wait_ns = WAIT_NS) {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        red_release_u32(count, 1u);
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(count) < target) {
            if (ld_acquire_u32(err) != 0u) break;  // another block gave up
            if (global_ns() - t0 > wait_ns) {
                atomicExch(err, 1u);
                on_timeout();
                break;
            }
        }
    }
    __syncthreads();
}

}  // namespace grid_dev
