// Device helpers shared by the library's kernels: timer, acquire loads, a
// grid-wide barrier with a deadline, warp reductions.
#pragma once

#include <climits>

#include "pic_internal.h"

namespace pic {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
    return *(volatile const unsigned*)p;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Grid-wide barrier for a cooperative (co-resident) launch.  Sense is kept in a
// generation counter.  A CTA that waits past `deadline` (globaltimer ns) records
// PIC_ERR_TIMEOUT and stops waiting; every CTA then sees the error and leaves.
// Returns the same boolean to every thread of the CTA.
__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned long long deadline) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nblocks = gridDim.x;
        unsigned gen = ld_acquire_u32(&c->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            while (ld_acquire_u32(&c->bar_gen) == gen) {
                if (ld_volatile(&c->err)) break;
                if (globaltimer_ns() > deadline) {
                    atomicCAS(&c->err, 0, (int)PIC_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        s_ok = ld_volatile(&c->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace pic
